// Transport sweep kernels: the upwind inversion of the streaming-plus-collision operator for every
// discrete ordinate (L^-1 of Section 2.1.1, L00^-1 of Section 3.2, Ltilde00^-1 of Section 3.3.2), with the
// angular reduction fused into the sweep.
//
// Work decomposition.  The mesh is cut into strips of 32 rows (in the sweep direction of a quadrant).  One
// CTA owns one (quadrant, angle group, strip); its warps hold disjoint directions of the group, APW each.
// Lane k of a warp owns row k of the strip and at step t solves the cell in column t - k, so the cell below
// (row k-1, same column) was solved by lane k-1 at step t-1 and arrives by a warp shuffle, and the cell to
// the left is the lane's own previous result.  Steps are grouped in chunks of kChunk:
//   - the cell data of the next chunk (source moments and sigma_t h, prepared once per sweep by
//     prep_kernel) is copied into shared memory with cp.async while the current chunk computes;
//   - each warp reads the chunk's inflow traces for its own directions from the strip below (prefetched
//     during the previous chunk) and stages them in shared memory; a trace that has not been written yet
//     still holds the empty pattern and is polled (bounded) until it arrives -- each warp depends only on
//     the warp with the same directions in the strip below, with no flags and no fences;
//   - per-step partial reductions go to a double-buffered shared array, and one barrier per chunk precedes
//     a fixed-order sum over the warps.
// CTAs take their (strip, quadrant, group) from an atomic ticket in strip-major order, so a CTA only waits
// for a strip owned by a CTA that started earlier: the wavefront cannot deadlock whatever the residency.
// Every wait is bounded (spin_limit polls); on expiry the CTA raises the error word and returns.
//
// Local coordinates.  Each quadrant is swept with the mesh mirrored so that its directions have
// Omega_x, Omega_y > 0; a cell's Legendre coefficients transform as (u0, sx u1, sy u2, sx sy u3).  With
// a = |Omega_x|, b = |Omega_y|, sigma-hat = sigma_t h, the per-cell Q1 block of L (eq-Ljk, times 2/h) is
//   [ 2(a+b+s)   2a              2b              0                  ]
//   [ -2a        2a+2/3(b+s)     0               2/3 b              ]
//   [ -2b        0               2b+2/3(a+s)     2/3 a              ]
//   [ 0          -2/3 b          -2/3 a          2/3(a+b)+2/9 s     ]
// and the upwind neighbours enter through their outflow traces: left face (U0 + U1 eta) with U0 = u0 + u1,
// U1 = u2 + u3; bottom face (V0 + V1 xi) with V0 = u0 + u2, V1 = u1 + u3.
//
// Reductions per cell (summed over the group's directions in a fixed order, one partial per quadrant-group):
//   LMDG_STD : P psi = sum w psi                                  (4 moments)
//   LMDG_LM  : P0 psi0 and the direction-dependent part of sum_l w_l L_l(u_l; b_r), r = 1..3 (u_l the full
//              per-direction trial function)
//   LMDG_RLM : as LM, plus P1 R psi0 (2 slope moments)
// from which the epilogue forms the reduced operator (see epilogue_kernel).  In the low-memory schemes the
// slopes of u_l are the isotropic X_1..3 (plus the reconstruction): their terms in L_l(u_l; b_r) that involve
// only the cell itself are a quadrature moment times the cell's slopes, added once per cell by the epilogue;
// the terms through the slope traces of the upwind cells (the same for every direction of LMDG) are summed
// once per lane and warp.  What remains per direction is the row-0 solve and the face terms of u0.
#include "lmdg_internal.h"

namespace lmdg {

namespace {

// Reciprocal by Newton's iteration r <- r (2 - x r) from a single-precision seed: each step squares the
// relative error, so two steps take the seed's ~2^-23 to below double rounding.
__device__ __forceinline__ double rcp(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
// FP32 sweeps (the inner solves of the refinement) take the hardware reciprocal approximation (rcp.approx, about
// one ulp) instead of the correctly rounded one.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// asynchronous global -> shared copies (16, 8 or 4 bytes, both addresses aligned to the size)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T> __device__ __forceinline__ void copy_cell(T *dst4, T *dsth, const T *src4, const T *srch);
template <> __device__ __forceinline__ void copy_cell<float>(float *d4, float *dh, const float *s4, const float *sh) {
  cp_async16(d4, s4);
  cp_async4(dh, sh);
}
template <> __device__ __forceinline__ void copy_cell<double>(double *d4, double *dh, const double *s4,
                                                             const double *sh) {
  cp_async16(d4, s4);
  cp_async16(d4 + 2, s4 + 2);
  cp_async8(dh, sh);
}
template <> __device__ __forceinline__ void copy_cell<f2>(f2 *d4, f2 *dh, const f2 *s4, const f2 *sh) {
  cp_async16(d4, s4);
  cp_async16(d4 + 2, s4 + 2);
  cp_async8(dh, sh);
}

// NR consecutive values (a cell's reduced moments) moved with the widest aligned vector accesses: the buffers
// hold them at NR-element strides, so NR = 4 floats are 16-byte aligned, NR = 6 floats 8-byte aligned and
// doubles and float-float pairs (NR even) 16-byte aligned.
template <typename T, int NR> __device__ __forceinline__ void store_nr(T *dst, const T *v) {
  if constexpr (is_f2<T>::value) {
#pragma unroll
    for (int q = 0; q < NR; q += 2)
      *reinterpret_cast<float4 *>(dst + q) = make_float4(v[q].hi, v[q].lo, v[q + 1].hi, v[q + 1].lo);
  } else if constexpr (sizeof(T) == 4 && NR % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NR; q += 4) *reinterpret_cast<float4 *>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < NR; q += 2) {
      if constexpr (sizeof(T) == 4) *reinterpret_cast<float2 *>(dst + q) = make_float2(v[q], v[q + 1]);
      else *reinterpret_cast<double2 *>(dst + q) = make_double2(v[q], v[q + 1]);
    }
  }
}
template <typename T, int NR> __device__ __forceinline__ void load_nr(T *dst, const T *src) {
  if constexpr (is_f2<T>::value) {
#pragma unroll
    for (int q = 0; q < NR; q += 2) {
      const float4 t = *reinterpret_cast<const float4 *>(src + q);
      dst[q] = f2(t.x, t.y); dst[q + 1] = f2(t.z, t.w);
    }
  } else if constexpr (sizeof(T) == 4 && NR % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NR; q += 4) {
      const float4 t = *reinterpret_cast<const float4 *>(src + q);
      dst[q] = t.x; dst[q + 1] = t.y; dst[q + 2] = t.z; dst[q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NR; q += 2) {
      if constexpr (sizeof(T) == 4) {
        const float2 t = *reinterpret_cast<const float2 *>(src + q);
        dst[q] = t.x; dst[q + 1] = t.y;
      } else {
        const double2 t = *reinterpret_cast<const double2 *>(src + q);
        dst[q] = t.x; dst[q + 1] = t.y;
      }
    }
  }
}
template <typename T, int NR> __device__ __forceinline__ void add_nr(T *acc, const T *src) {
  if constexpr (is_f2<T>::value) {
#pragma unroll
    for (int q = 0; q < NR; q += 2) {
      const float4 t = *reinterpret_cast<const float4 *>(src + q);
      acc[q] += f2(t.x, t.y); acc[q + 1] += f2(t.z, t.w);
    }
  } else if constexpr (sizeof(T) == 4 && NR % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NR; q += 4) {
      const float4 t = *reinterpret_cast<const float4 *>(src + q);
      acc[q] += t.x; acc[q + 1] += t.y; acc[q + 2] += t.z; acc[q + 3] += t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NR; q += 2) {
      if constexpr (sizeof(T) == 4) {
        const float2 t = *reinterpret_cast<const float2 *>(src + q);
        acc[q] += t.x; acc[q + 1] += t.y;
      } else {
        const double2 t = *reinterpret_cast<const double2 *>(src + q);
        acc[q] += t.x; acc[q + 1] += t.y;
      }
    }
  }
}

// the four Legendre coefficients of a standard-scheme cell: one 16-byte store (float) or two (double)
template <typename T> __device__ __forceinline__ void store_psi4(void *psi, size_t idx, T a, T b, T c, T d) {
  if constexpr (std::is_same<T, float>::value) {
    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(psi) + idx) = make_float4(a, b, c, d);
  } else if constexpr (std::is_same<T, double>::value) {
    double2 *p = reinterpret_cast<double2 *>(reinterpret_cast<double *>(psi) + idx);
    p[0] = make_double2(a, b);
    p[1] = make_double2(c, d);
  } else {
    float *p = reinterpret_cast<float *>(psi) + idx;   // float-float sweeps do not store (the host refuses it)
    p[0] = a.hi; p[1] = b.hi; p[2] = c.hi; p[3] = d.hi;
  }
}
template <typename T> __device__ __forceinline__ void store_psi0(void *psi, size_t idx, T v, int bf16) {
  if constexpr (is_f2<T>::value) {
    reinterpret_cast<float *>(psi)[idx] = v.hi;   // float-float sweeps do not store (the host refuses it)
  } else {
    if (bf16) reinterpret_cast<__nv_bfloat16 *>(psi)[idx] = __float2bfloat16((float)v);
    else reinterpret_cast<T *>(psi)[idx] = v;
  }
}

constexpr unsigned kFull = 0xffffffffu;

// Polling of a strip trace that has not arrived: sleeps doubling from kPollNsMin to kPollNsMax between polls (a
// trace is late by a fraction of a chunk in the steady wavefront, by hundreds of steps while it fills), and a
// look at the error word every kAbortEvery polls.
#ifndef LMDG_POLL_NS_MAX
#define LMDG_POLL_NS_MAX 256
#endif
constexpr unsigned kPollNsMin = 16, kPollNsMax = LMDG_POLL_NS_MAX;
constexpr long long kAbortEvery = 64;

// Strip-boundary traces carry their own readiness: the buffer holds the NaN pattern kTraceEmpty (every 32-bit
// word 0xFFF7FFF7, never produced by arithmetic, whose NaNs are canonical) until the producing lane stores
// the value, and the consuming warp writes the pattern back after reading it.  Aligned 32/64-bit stores are
// single-copy atomic, so a reader sees either the pattern or the whole value.
__device__ __forceinline__ bool is_empty(float v) { return __float_as_uint(v) == kTraceEmpty; }
__device__ __forceinline__ bool is_empty(double v) {
  return (unsigned long long)__double_as_longlong(v) == (((unsigned long long)kTraceEmpty << 32) | kTraceEmpty);
}
__device__ __forceinline__ bool is_empty(f2 v) {
  return __float_as_uint(v.hi) == kTraceEmpty && __float_as_uint(v.lo) == kTraceEmpty;
}
__device__ __forceinline__ float empty_value(float) { return __uint_as_float(kTraceEmpty); }
__device__ __forceinline__ f2 empty_value(f2) { return f2(__uint_as_float(kTraceEmpty), __uint_as_float(kTraceEmpty)); }
__device__ __forceinline__ double empty_value(double) {
  return __longlong_as_double((long long)(((unsigned long long)kTraceEmpty << 32) | kTraceEmpty));
}
__device__ __forceinline__ float ld_relaxed_t(const float *p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed_t(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
// a float-float trace moves as one 64-bit word (hi in the low half), so that it is read and written whole
__device__ __forceinline__ f2 ld_relaxed_t(const f2 *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return f2(__uint_as_float((unsigned)v), __uint_as_float((unsigned)(v >> 32)));
}
// Trace stores are relaxed at GPU scope, like the polling loads, so the data-carried readiness protocol is
// race-free in the PTX memory model (a weak store paired with a relaxed load would be a data race there).
__device__ __forceinline__ void st_trace(float *p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}
__device__ __forceinline__ void st_trace(double *p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void st_trace(f2 *p, f2 v) {
  const unsigned long long b =
      ((unsigned long long)__float_as_uint(v.lo) << 32) | (unsigned long long)__float_as_uint(v.hi);
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b));
}

// Sign flip by the bit pattern (an integer op instead of an FP64 multiply): m = 0 keeps v, m = 0x80000000 negates.
__device__ __forceinline__ double flip(double v, unsigned m) {
  return __hiloint2double(__double2hiint(v) ^ (int)m, __double2loint(v));
}
__device__ __forceinline__ float flip(float v, unsigned m) { return __uint_as_float(__float_as_uint(v) ^ m); }
__device__ __forceinline__ f2 flip(f2 v, unsigned m) { return f2(flip(v.hi, m), flip(v.lo, m)); }

template <typename T> __device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(kFull, v, 1); }
template <> __device__ __forceinline__ f2 shfl_up1<f2>(f2 v) {
  return f2(__shfl_up_sync(kFull, v.hi, 1), __shfl_up_sync(kFull, v.lo, 1));
}
// read-only load of a coefficient-table entry
template <typename T> __device__ __forceinline__ T tload(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ f2 tload<f2>(const f2 *p) {
  const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
  return f2(t.x, t.y);
}

// With coefficient tables the sigma_t h slot of the staged cell data carries the material index as a bit pattern.
__device__ __forceinline__ double mat_bits(int m, double) { return __longlong_as_double((long long)m); }
__device__ __forceinline__ float mat_bits(int m, float) { return __int_as_float(m); }
__device__ __forceinline__ f2 mat_bits(int m, f2) { return f2(__int_as_float(m), 0.0f); }
__device__ __forceinline__ int mat_of(double v) { return (int)__double_as_longlong(v); }
__device__ __forceinline__ int mat_of(float v) { return __float_as_int(v); }
__device__ __forceinline__ int mat_of(f2 v) { return __float_as_int(v.hi); }

}  // namespace

// Shared-memory bytes of one CTA: partial reductions [2][kChunk][W][32][NR], cell data [2][kChunk][32][4] and
// [2][kChunk][32], upstream traces [W][APW][kChunk][NS], RLMDG suppression bits [2][kChunk][32].
template <typename T>
size_t sweep_smem_bytes(int variant, int warps, int apw) {
  const int NR = nr_of(variant);
  const int NS = ns_of(variant);
  return sizeof(T) * ((size_t)2 * kChunk * warps * NR * 32 + (size_t)2 * kChunk * 32 * 5 +
                      (size_t)warps * apw * kChunk * NS) +
         sizeof(unsigned) * (size_t)2 * kChunk * 32;
}

// Per-cell inputs of one sweep, global basis: src = 2h D_r (sigma_s/eps X_r + eps q_r) for the standard
// scheme; (2h (sigma_s/eps X0 + eps q0), isotropic slopes -(X1 + P1 r_alpha)) for the low-memory schemes
// (q and P1 r_alpha only in source sweeps; angle-dependent q is added inside the sweep).  sh = sigma_t h.
template <typename T, int VAR>
__global__ void prep_kernel(int nx, T h, T eps, const double *__restrict__ X, const T *__restrict__ sse,
                            const T *__restrict__ sigt, const T *__restrict__ q, const T *__restrict__ p1ra,
                            int source, int q_iso, T *__restrict__ src, T *__restrict__ sh,
                            const int *__restrict__ mat) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  const double2 Xa = reinterpret_cast<const double2 *>(X)[2 * (size_t)K];
  const double2 Xb = reinterpret_cast<const double2 *>(X)[2 * (size_t)K + 1];
  const T s = sse[K];
  T q4[4] = {0, 0, 0, 0};
  if (source && q_iso) {
    const T *qp = q + 4 * (size_t)K;
    q4[0] = qp[0]; q4[1] = qp[1]; q4[2] = qp[2]; q4[3] = qp[3];
  }
  T o[4];
  if (VAR == 0) {
    o[0] = 2 * h * (s * (T)Xa.x + eps * q4[0]);
    o[1] = (2 * h / 3) * (s * (T)Xa.y + eps * q4[1]);
    o[2] = (2 * h / 3) * (s * (T)Xb.x + eps * q4[2]);
    o[3] = (2 * h / 9) * (s * (T)Xb.y + eps * q4[3]);
  } else if (VAR == kP0) {
    o[0] = 2 * h * (s * (T)Xa.x + eps * q4[0]);
    o[1] = 0; o[2] = 0; o[3] = 0;
  } else {
    T p1 = 0, p2 = 0;
    T p3 = 0;
    if (VAR >= 2 && source && p1ra) {
      p1 = p1ra[3 * (size_t)K]; p2 = p1ra[3 * (size_t)K + 1]; p3 = p1ra[3 * (size_t)K + 2];
    }
    o[0] = 2 * h * (s * (T)Xa.x + eps * q4[0]);
    o[1] = -((T)Xa.y + p1);
    o[2] = -((T)Xb.x + p2);
    o[3] = -((T)Xb.y + p3);
  }
  T *d = src + 4 * (size_t)K;
  d[0] = o[0]; d[1] = o[1]; d[2] = o[2]; d[3] = o[3];
  sh[K] = mat ? mat_bits(mat[K], (T)0) : sigt[K] * h;
}

// Coefficients of the element solves for one material (s = sigma_t h) and one direction class (a, b) =
// (|Omega_x|, |Omega_y|), in the local frame of the kernel, with d0 = 2(a + b + s), d1 = 2a + 2/3 (b + s),
// d2 = 2b + 2/3 (a + s), d3 = 2/3 (a + b) + 2/9 s:
//   standard: i1 = 1/d1, i2 = 1/d2, p1 = 2a i1, p2 = 2b i2, q1 = 2/3 b i1, q2 = 2/3 a i2, and with the 2x2 Schur
//             system (a00 a03; a03 a33) of the (u0, u3) unknowns, c0 = a33/det, c1 = a03/det, c3 = a00/det;
//   LMDG: 1/d0;
//   RLMDG: 1/(d0 + cx + cy) with cx = a for a reconstructed x slope, 2a on an inflow x face, 0 where the
//          reconstruction is suppressed (likewise cy), at index (x state) + 3 (y state), states in that order;
//   RLMDG*: the same with cx = 3a/2 for the three-cell slope, 2a on an inflow face, a in the second cell;
//   P0-DG: 1/d0 as LMDG.
int coef_count(int variant) { return (variant == LMDG_LM || variant == kP0) ? 1 : 9; }

__global__ void coef_kernel(int variant, int nmat, int ncls, const double *__restrict__ matsh,
                            const double *__restrict__ cls_ab, double *__restrict__ coef) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nmat * ncls) return;
  const int m = id / ncls, c = id - m * ncls;
  const double s = matsh[m], a = cls_ab[2 * c], b = cls_ab[2 * c + 1];
  const double c23 = 2.0 / 3.0, c29 = 2.0 / 9.0;
  const double d0 = 2 * (a + b + s), d1 = 2 * a + c23 * (b + s), d2 = 2 * b + c23 * (a + s), d3 = c23 * (a + b) + c29 * s;
  if (variant == LMDG_STD) {
    double *o = coef + (size_t)id * 9;
    const double i1 = 1.0 / d1, i2 = 1.0 / d2;
    const double a00 = d0 + 4 * a * a * i1 + 4 * b * b * i2;
    const double a03 = -(4.0 / 3.0) * a * b * (i1 + i2);
    const double a33 = d3 + (4.0 / 9.0) * (b * b * i1 + a * a * i2);
    const double det = a00 * a33 - a03 * a03;
    o[0] = i1; o[1] = i2; o[2] = 2 * a * i1; o[3] = 2 * b * i2; o[4] = c23 * b * i1; o[5] = c23 * a * i2;
    o[6] = a33 / det; o[7] = a03 / det; o[8] = a00 / det;
  } else if (variant == LMDG_LM || variant == kP0) {
    coef[id] = 1.0 / d0;
  } else {
    double *o = coef + (size_t)id * 9;
    const bool star = variant == kRlmStar;
    const double cx[3] = {star ? 1.5 * a : a, 2 * a, star ? a : 0.0};
    const double cy[3] = {star ? 1.5 * b : b, 2 * b, star ? b : 0.0};
    for (int ys = 0; ys < 3; ++ys)
      for (int xs = 0; xs < 3; ++xs) o[xs + 3 * ys] = 1.0 / (d0 + cx[xs] + cy[ys]);
  }
}

cudaError_t build_coef_tables(int variant, int nmat, int ncls, const double *matsh, const double *cls_ab,
                              double *coef, cudaStream_t s) {
  const int tot = nmat * ncls;
  add_launches(1);
  coef_kernel<<<(tot + 255) / 256, 256, 0, s>>>(variant, nmat, ncls, matsh, cls_ab, coef);
  return cudaGetLastError();
}

// Minimum resident CTAs per SM requested from the compiler for the FP32 instances (register budget).
#ifndef LMDG_MINB32
#define LMDG_MINB32 2
#endif

// TAB: the element-solve coefficients come from the FP64 tables (per material and direction class; FP64
// instances only), else they are formed in the kernel from sigma_t h.  LEAN: a non-storing sweep without inflow
// data, angle-dependent source or correlation (the GMRES iterations; the residual sweeps of problems with vacuum
// inflow and isotropic source), compiled without the per-step tests for them (FP32 and float-float instances).
// LSTORE (with LEAN; FP32, one or two directions per warp): the same sweep storing the angular unknowns
// unconditionally -- the recovery sweep of a vacuum, isotropic-source problem.
template <typename T, int VAR, int APW, bool TAB, bool LEAN, bool LSTORE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? LMDG_MINB32 : 1) sweep_kernel(const SweepArgs<T> A) {
  constexpr bool P0 = VAR == kP0;         // P0-DG: the LMDG row-0 solve without slopes
  constexpr bool Q1R = VAR == kRlmQ1;     // RLMDG with the Q1-type reconstruction (the xi eta term)
  constexpr int NR = nr_of(VAR);          // reduced values per cell
  constexpr int NS = ns_of(VAR);          // trace values passed downwind per face
  constexpr int NC = (VAR == 1 || P0) ? 1 : 9;   // table coefficients per (material, class)
  constexpr int C = kChunk;
  // the adjoint correlation exists for the FP64 instances only (compiled out of FP32)
  constexpr bool kF64 = std::is_same<T, double>::value;
  const bool use_corr = kF64 && !LEAN && A.corr != nullptr;
  const bool local = kF64 && !LEAN && A.local != 0;   // cut the upwind coupling (diagonal blocks of K)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_unit, s_abort;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = A.g.warps;
  const int ni = A.ni, nj = A.nj, nx = A.nx;   // ni columns along x, nj rows along y, nx cells
  const int nfaces = 2 * (ni + nj);               // inflow data per direction: west, east (nj each), south, north (ni)
  T *red = reinterpret_cast<T *>(smem_raw);          // [2][C][W][32][NR]
  T *cs = red + (size_t)2 * C * W * NR * 32;         // [2][C][32][4]
  T *csh = cs + (size_t)2 * C * 32 * 4;              // [2][C][32]
  T *yup = csh + (size_t)2 * C * 32;                 // [W][APW][C][NS]
  unsigned *csup = reinterpret_cast<unsigned *>(yup + (size_t)W * APW * C * NS);   // [2][C][32]

  if (threadIdx.x == 0) {
    s_unit = (int)atomicAdd(&A.ctrl[0], 1u);
    s_abort = 0;
  }
  __syncthreads();
  const int unit = s_unit;
  const int per_strip = A.npq;                      // partial sets of this launch (tickets strip-major)
  const int strip = unit / per_strip;
  const int pq = A.pq0 + (unit - strip * per_strip);   // partial index = quadrant * groups + group
  const int quad = pq / A.g.groups, grp = pq - quad * A.g.groups;
  const int sx = (quad == 0 || quad == 3) ? 1 : -1;
  const int sy = (quad <= 1) ? 1 : -1;
  const unsigned mx = sx > 0 ? 0u : 0x80000000u, my = sy > 0 ? 0u : 0x80000000u, mxy = mx ^ my;
  const int gsize = (A.nq + A.g.groups - 1) / A.g.groups;
  const int g0 = grp * gsize;
  const int gcount = min(gsize, A.nq - g0);
  // warps holding at least one direction (warp w holds directions w, w + W, ...); the others only stage data
  // and take part in the barriers -- they skip the steps and the chunk sum leaves their slots out
  const int Wact = min(W, gcount);
  const T c23 = (T)(2.0 / 3.0), c29 = (T)(2.0 / 9.0);

  // per-direction constants (signs of the quadrant folded in: the reduction is in the global frame)
  int ang[APW], uA[APW], cA[APW], kA[APW];
  T wA[APW], aA[APW], bA[APW], c2a[APW], c2b[APW], c23a[APW], c23b[APW];
  T Wx[APW], Wy[APW];                 // w sx (2a, ...) / w sy (2b, ...): face terms of u0 (LM, RLM); w sx, w sy (STD)
  T Dx[APW], Dy[APW], nWxb[APW], nWya[APW], W3a[APW], W3b[APW], wx[APW], wy[APW], wxy[APW];   // RLMDG; W3*: w sx sy
                                                                                           // (STD)
  int nA = 0;
  T Ga = 0, Gb = 0;                   // LMDG: sum over the warp's directions of w 2/3 a, w 2/3 b
#pragma unroll
  for (int k = 0; k < APW; ++k) {
    const int idx = warp + k * W;
    ang[k] = quad * A.nq + g0 + min(idx, gcount - 1);
    if (idx < gcount) nA = k + 1;
    uA[k] = A.perm[ang[k]];
    cA[k] = (kF64 && A.corr) ? A.rev[ang[k]] : 0;
    kA[k] = TAB ? A.cls[ang[k]] * NC : 0;
    const T w = A.pd.w[ang[k]], a = fabs(A.pd.ox[ang[k]]), b = fabs(A.pd.oy[ang[k]]);
    wA[k] = w; aA[k] = a; bA[k] = b;
    c2a[k] = 2 * a; c2b[k] = 2 * b; c23a[k] = c23 * a; c23b[k] = c23 * b;
    if (VAR == 0) {
      Wx[k] = flip(w, mx); Wy[k] = flip(w, my); W3a[k] = flip(w, mxy);
    } else {
      Wx[k] = flip(2 * w * a, mx); Wy[k] = flip(2 * w * b, my);
      if (idx < gcount) { Ga += w * c23 * a; Gb += w * c23 * b; }
    }
    if (VAR >= 2 && !P0) {
      Dx[k] = flip(w * (2 * a + c23 * b), mx); Dy[k] = flip(w * (2 * b + c23 * a), my);
      nWxb[k] = flip(w * c23 * b, mx ^ 0x80000000u); nWya[k] = flip(w * c23 * a, my ^ 0x80000000u);
      W3a[k] = flip(w * c23 * a, mxy); W3b[k] = flip(w * c23 * b, mxy);
      wx[k] = flip(w, mx); wy[k] = flip(w, my); wxy[k] = flip(w, mxy);
    }
  }
  // LMDG slope-trace terms, per lane: -sx Gb V1 (r = 1), -sy Ga U1 (r = 2), sx sy (Ga U1 + Gb V1) (r = 3)
  const T nGb = flip(Gb, mx ^ 0x80000000u), nGa = flip(Ga, my ^ 0x80000000u);
  const T G3a = flip(Ga, mxy), G3b = flip(Gb, mxy);

  const int row = strip * 32 + lane;
  const bool row_ok = row < nj;
  const int j = sy > 0 ? row : nj - 1 - row;
  const T h = A.h;
  const T *tab = TAB ? A.coef : nullptr;
  const int tab_stride = TAB ? A.ncls * NC : 0;

  // upwind state: xs = this lane's previous cell (the left neighbour), ys = what goes to the cell above
  //   STD: (U0, U1) / (V0, V1) outflow traces;  LM: mean traces (U0 / V0) per direction, the slope traces per
  //   lane (xl1 / yl1);  RLM: (U0, U1, u0) / (V0, V1, u0) per direction
  T xs[APW][NS], ys[APW][NS];
#pragma unroll
  for (int k = 0; k < APW; ++k)
#pragma unroll
    for (int c = 0; c < NS; ++c) xs[k][c] = ys[k][c] = (T)0;
  T xl1 = 0, yl1 = 0;

  const bool has_above = strip + 1 < A.g.strips;
  // upstream trace entry of item it = (direction k, step s, component c) of the chunk starting at t0
  constexpr int NI = (APW * C * NS + 31) / 32;
  auto up_addr = [&](int it, int t0) -> T * {
    if (it >= APW * C * NS) return nullptr;
    const int k = it / (C * NS), rem = it - k * C * NS, s = rem / NS, c = rem - s * NS;
    const int x = t0 + s;
    if (k >= nA || x >= ni) return nullptr;
    const int ak = quad * A.nq + g0 + min(warp + k * W, gcount - 1);
    return A.ytr + (((size_t)ak * A.g.strips + (strip - 1)) * ni + x) * kTraceStride + c;
  };
  T pre[NI];
#pragma unroll
  for (int q = 0; q < NI; ++q) pre[q] = (T)0;
  if (strip > 0) {
#pragma unroll
    for (int q = 0; q < NI; ++q) {
      const T *p = up_addr(lane + 32 * q, 0);
      if (p) pre[q] = ld_relaxed_t(p);
    }
  }
  const int nsteps = ni + 31;
  const int nchunks = (nsteps + C - 1) / C;
  const size_t plane = psi_plane(ni, nj);   // slots per direction of the stored psi

  // cell data of chunk cc -> buffer cc & 1 (item = (step, lane) of the chunk)
  auto stage = [&](int cc) {
    const int b = cc & 1;
    for (int it = threadIdx.x; it < C * 32; it += blockDim.x) {
      const int s = it >> 5, l = it & 31;
      const int r = strip * 32 + l, x = cc * C + s - l;
      if (r < nj && x >= 0 && x < ni) {
        const int ii = sx > 0 ? x : ni - 1 - x, jj = sy > 0 ? r : nj - 1 - r;
        const size_t K = (size_t)jj * ni + ii;
        copy_cell<T>(cs + ((size_t)(b * C + s) * 32 + l) * 4, csh + (size_t)(b * C + s) * 32 + l,
                     A.cellsrc + 4 * K, A.cellsh + K);
        if (VAR == 2 && A.supp) cp_async4(csup + (size_t)(b * C + s) * 32 + l, A.supp + K);
      }
    }
    cp_async_commit();
  };

  stage(0);
  cp_async_wait_all();
  __syncthreads();

  const bool src_bnd = !LEAN && A.source && A.pd.alpha;

  for (int cc = 0; cc < nchunks; ++cc) {
    const int t0 = cc * C;
    const int b = cc & 1;
    if (cc + 1 < nchunks) stage(cc + 1);

    // ---- inflow from the strip below: the traces of columns [t0, t0 + C) for this warp's directions
    // (prefetched during the previous chunk), polled until present, staged in shared memory, and consumed
    bool wabort = false;
    if (strip > 0 && t0 < ni) {
      int ab = 0;
      T *yw = yup + (size_t)warp * APW * C * NS;
#pragma unroll
      for (int q = 0; q < NI; ++q) {
        const int it = lane + 32 * q;
        T *p = up_addr(it, t0);
        if (p) {
          T v = pre[q];
          long long spins = 0;
          unsigned sleep_ns = kPollNsMin;
          while (is_empty(v)) {
            // the error word (one line every waiter on the GPU reads) is checked every kAbortEvery polls only
            ++spins;
            if (spins > A.spin_limit || ((spins & (kAbortEvery - 1)) == 0 && ld_relaxed(&A.ctrl[1]) != 0u)) {
              atomicExch(&A.ctrl[1], 1u);
              ab = 1;
              break;
            }
            __nanosleep(sleep_ns);
            if (sleep_ns < kPollNsMax) sleep_ns <<= 1;
            v = ld_relaxed_t(p);
          }
          yw[it] = v;
          st_trace(p, empty_value(v));
        }
      }
      wabort = __any_sync(kFull, ab) != 0;
      __syncwarp();
      if (wabort && lane == 0) s_abort = 1;
      if (!wabort && t0 + C < ni) {
#pragma unroll
        for (int q = 0; q < NI; ++q) {
          const T *p = up_addr(lane + 32 * q, t0 + C);
          if (p) pre[q] = ld_relaxed_t(p);
        }
      }
    }

    // ---- C steps of the diagonal pipeline
    if (!wabort && warp < Wact) {
      for (int s = 0; s < C; ++s) {
        const int t = t0 + s;
        if (t >= nsteps) break;
        const int x = t - lane;
        const bool act = row_ok && x >= 0 && x < ni;
        const int i = sx > 0 ? x : ni - 1 - x;
        const int K = act ? j * ni + i : 0;
        // stored angular unknowns in wavefront order (psi_slot): this step's 32 cells are consecutive slots, so a
        // warp's psi stores coalesce; the adjoint's correlation input is the opposite direction's plane, whose
        // frame is this one mirrored in both axes
        const size_t pslot = ((size_t)strip * nsteps + t) * 32 + lane;
        const size_t rslot = use_corr && act ? psi_slot(ni, ni - 1 - x, nj - 1 - row) : 0;
        const bool xbnd = (x == 0);
        const bool ybnd = (strip == 0 && lane == 0);
        const T *yws = yup + ((size_t)warp * APW * C + s) * NS;   // + k * C * NS: direction k's inflow (lane 0)
        // per-cell data in local coordinates
        const T *cp4 = cs + ((size_t)(b * C + s) * 32 + lane) * 4;
        const T S0 = cp4[0], A1 = flip(cp4[1], mx), A2 = flip(cp4[2], my), A3 = flip(cp4[3], mxy);
        const T st = csh[(size_t)(b * C + s) * 32 + lane];
        // RLMDG: upwind faces without reconstruction (the upwind side is west / south in the local frame)
        bool xsup = false, ysup = false;
        if (VAR == 2 && A.supp && act) {
          const unsigned mk = csup[(size_t)(b * C + s) * 32 + lane];
          xsup = (mk & (sx > 0 ? 1u : 2u)) != 0;
          ysup = (mk & (sy > 0 ? 4u : 8u)) != 0;
        }
        const T *cf = TAB ? tab + (size_t)mat_of(st) * tab_stride : nullptr;
        // RLMDG*: the reconstruction of this cell in x (and y) -- inflow cell, second cell (two-cell
        // difference) or interior (three-cell): slope = f0 u0 - f1 u_up + f2 u_upup, row-0 rhs gains
        // a (g1 u_up - g2 u_upup), table state 1 / 2 / 0
        T f0x = 0, f1x = 0, f2x = 0, g1x = 0, g2x = 0, f0y = 0, f1y = 0, f2y = 0, g1y = 0, g2y = 0, cdx = 0, cdy = 0;
        int stx = 0, sty = 0;
        if (VAR == 3) {
          if (xbnd) { stx = 1; f0x = 1; cdx = 2; }
          else if (x == 1) { stx = 2; f0x = (T)0.5; f1x = (T)0.5; g1x = 1; cdx = 1; }
          else { f0x = (T)0.75; f1x = 1; f2x = (T)0.25; g1x = 2; g2x = (T)0.5; cdx = (T)1.5; }
          if (ybnd) { sty = 1; f0y = 1; cdy = 2; }
          else if (row == 1) { sty = 2; f0y = (T)0.5; f1y = (T)0.5; g1y = 1; cdy = 1; }
          else { f0y = (T)0.75; f1y = 1; f2y = (T)0.25; g1y = 2; g2y = (T)0.5; cdy = (T)1.5; }
        }

        T acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = 0;

        // LMDG: the slope traces from below (one per lane; every direction carries the same value)
        T yl1_in = 0;
        if (VAR == 1) {
          yl1_in = shfl_up1(yl1);
          if (lane == 0) yl1_in = (ybnd || nA == 0) ? (T)0 : yws[1];
          if (local) { yl1_in = 0; xl1 = 0; }
        }
        const T A13 = A1 + A3, A23 = A2 + A3;

#pragma unroll
        for (int k = 0; k < APW; ++k) {
          if (k < nA) {
            // inflow from the cell below (LMDG: the mean trace only; its slope trace is per lane)
            constexpr int NSH = (VAR == 1 || P0) ? 1 : NS;
            T yin[NS];
#pragma unroll
            for (int c = 0; c < NSH; ++c) yin[c] = shfl_up1(ys[k][c]);
            if (act) {
              if (lane == 0) {
#pragma unroll
                for (int c = 0; c < NSH; ++c) yin[c] = ybnd ? (T)0 : yws[(size_t)k * C * NS + c];
              }
              if (local) {
#pragma unroll
                for (int c = 0; c < NS; ++c) { yin[c] = 0; xs[k][c] = 0; }
              }
              const T a = aA[k], bb = bA[k], wl = wA[k];
              // inflow boundary data (source sweeps): left face on x == 0, bottom face on the first row
              T xa0 = 0, xa1 = 0, ya0 = 0, ya1 = 0;
              if (src_bnd) {
                if (xbnd) {
                  const T *ap = A.pd.alpha + ((size_t)ang[k] * nfaces + (sx > 0 ? 0 : nj) + j) * 2;
                  xa0 = ap[0];
                  xa1 = flip(ap[1], my);
                }
                if (ybnd) {
                  const T *ap = A.pd.alpha + ((size_t)ang[k] * nfaces + 2 * nj + (sy > 0 ? 0 : ni) + i) * 2;
                  ya0 = ap[0];
                  ya1 = flip(ap[1], mx);
                }
              }
              T S = S0;
              const T *qp = nullptr;
              if (!LEAN && A.source && A.q_per_angle) {
                qp = A.pd.q + ((size_t)ang[k] * nx + K) * 4;
                S += 2 * h * A.eps * qp[0];
              }
              if constexpr (VAR == 0) {
                // ---------------- standard Q1 block solve; inflow traces vanish outside the mesh
                T sa1 = A1, sa2 = A2, sa3 = A3;
                if (qp) {
                  const T e = A.eps;
                  sa1 += flip((2 * h / 3) * e * qp[1], mx);
                  sa2 += flip((2 * h / 3) * e * qp[2], my);
                  sa3 += flip((2 * h / 9) * e * qp[3], mxy);
                }
                T U0 = xs[k][0], U1 = xs[k][1], V0 = yin[0], V1 = yin[1];
                if (src_bnd) { U0 += xa0; U1 += xa1; V0 += ya0; V1 += ya1; }
                const T ca = c23a[k], cb = c23b[k];
                const T r0 = S + c2a[k] * U0 + c2b[k] * V0;
                const T r1 = sa1 - c2a[k] * U0 + cb * V1;
                const T r2 = sa2 + ca * U1 - c2b[k] * V0;
                const T r3 = sa3 - ca * U1 - cb * V1;
                T u0, u1, u2, u3;
                if (TAB) {
                  const T *cfk = cf + kA[k];
                  const T i1 = tload(cfk), i2 = tload(cfk + 1), p1 = tload(cfk + 2), p2 = tload(cfk + 3);
                  const T q1 = tload(cfk + 4), q2 = tload(cfk + 5), e0 = tload(cfk + 6), e1 = tload(cfk + 7);
                  const T e3 = tload(cfk + 8);
                  const T b0 = r0 - p1 * r1 - p2 * r2;
                  const T b3 = r3 + q1 * r1 + q2 * r2;
                  u0 = e0 * b0 - e1 * b3;
                  u3 = e3 * b3 - e1 * b0;
                  u1 = i1 * r1 + p1 * u0 - q1 * u3;
                  u2 = i2 * r2 + p2 * u0 - q2 * u3;
                } else {
                  const T d0 = 2 * (a + bb + st);
                  const T d1 = 2 * a + c23 * (bb + st);
                  const T d2 = 2 * bb + c23 * (a + st);
                  const T d3 = c23 * (a + bb) + c29 * st;
                  const T i1 = rcp(d1), i2 = rcp(d2);
                  const T a00 = d0 + 4 * a * a * i1 + 4 * bb * bb * i2;
                  const T a03 = -(T)(4.0 / 3.0) * a * bb * (i1 + i2);
                  const T a33 = d3 + (T)(4.0 / 9.0) * (bb * bb * i1 + a * a * i2);
                  const T b0 = r0 - 2 * a * r1 * i1 - 2 * bb * r2 * i2;
                  const T b3 = r3 + c23 * (bb * r1 * i1 + a * r2 * i2);
                  const T idet = rcp(a00 * a33 - a03 * a03);
                  u0 = (a33 * b0 - a03 * b3) * idet;
                  u3 = (a00 * b3 - a03 * b0) * idet;
                  u1 = (r1 + 2 * a * u0 - c23 * bb * u3) * i1;
                  u2 = (r2 + 2 * bb * u0 - c23 * a * u3) * i2;
                }
                if (use_corr) {
                  // adjoint correlation: this sweep's psi (the multiplier of the opposite direction) times the
                  // stored forward psi of that opposite direction, per Legendre moment
                  const double *pf = A.corr + ((size_t)cA[k] * plane + rslot) * 4;
                  acc[0] += wl * u0 * (T)pf[0];
                  acc[1] += Wx[k] * u1 * (T)pf[1];
                  acc[2] += Wy[k] * u2 * (T)pf[2];
                  acc[3] += W3a[k] * u3 * (T)pf[3];
                } else if (k == 0) {   // the first direction sets the sums (no addition of zero)
                  acc[0] = wl * u0;
                  acc[1] = Wx[k] * u1;
                  acc[2] = Wy[k] * u2;
                  acc[3] = W3a[k] * u3;
                } else {
                  acc[0] += wl * u0;
                  acc[1] += Wx[k] * u1;
                  acc[2] += Wy[k] * u2;
                  acc[3] += W3a[k] * u3;
                }
                xs[k][0] = u0 + u1; xs[k][1] = u2 + u3;
                ys[k][0] = u0 + u2; ys[k][1] = u1 + u3;
                if (LSTORE || (!LEAN && A.psi)) store_psi4<T>(A.psi, ((size_t)uA[k] * plane + pslot) * 4, u0, flip(u1, mx), flip(u2, my),
                                         flip(u3, mxy));
              } else if constexpr (VAR == 1 || P0) {
                // ---------------- LMDG: row 0 of L00 for u0; u1..3 = A1..3 (isotropic)
                //   rhs = S + 2a (U0 - A1) + 2b (V0 - A2), U0 / V0 the mean inflow traces (alpha on the boundary)
                const T U0 = xs[k][0], V0 = yin[0];
                T rhs = c2a[k] * (U0 - A1) + (c2b[k] * (V0 - A2) + S);
                if (src_bnd) rhs += c2a[k] * xa0 + c2b[k] * ya0;
                const T u0 = rhs * (TAB ? tload(cf + kA[k]) : rcp(2 * (a + bb + st)));
                // direction-dependent part of L(u; b_1), L(u; b_2): 2a (U0 - u0), 2b (V0 - u0) (zero inflow traces
                // outside the mesh)
                if (use_corr) {
                  acc[0] += wl * u0 * (T)A.corr[(size_t)cA[k] * plane + rslot];
                } else {
                  acc[0] = fma(wl, u0, acc[0]);
                  if constexpr (!P0) {
                    acc[1] = fma(Wx[k], U0 - u0, acc[1]);
                    acc[2] = fma(Wy[k], V0 - u0, acc[2]);
                  }
                }
                if constexpr (P0) {
                  xs[k][0] = u0;
                  ys[k][0] = u0;
                } else {
                  xs[k][0] = u0 + A1;
                  ys[k][0] = u0 + A2;
                  ys[k][1] = A13;
                }
                if (LSTORE || (!LEAN && A.psi)) store_psi0<T>(A.psi, (size_t)uA[k] * plane + pslot, u0, A.psi_bf16);
              } else {
                // ---------------- RLMDG: row 0 of Ltilde00 with the upwind reconstruction
                //   slopes (h/2) delta of u0: (u0 - u0_up)/2 inside, u0 - alpha_mid on an inflow face, 0 across
                //   a suppressed face; 2a (h/2) delta_x enters row 0 through L01.  RLMDG*: the three-cell slope
                //   (3 u0 - 4 u0_up + u0_upup)/4 from the third cell on
                const T U0 = xs[k][0], U1 = xs[k][1], Ux = xs[k][2];
                const T V0 = yin[0], V1 = yin[1], Vy = yin[2];
                T rhs = c2a[k] * (U0 - A1) + (c2b[k] * (V0 - A2) + S);
                T u0, rec1, rec2;
                if constexpr (VAR == 3) {
                  const T Uxx = xs[k][3], Vyy = yin[3];
                  rhs = fma(a, g1x * Ux - g2x * Uxx, fma(bb, g1y * Vy - g2y * Vyy, rhs));
                  if (src_bnd) rhs += 4 * (a * xa0 + bb * ya0);
                  const T inv = TAB ? tload(cf + kA[k] + stx + 3 * sty)
                                    : rcp(2 * st + a * (2 + cdx) + bb * (2 + cdy));
                  u0 = rhs * inv;
                  rec1 = f0x * u0 - (f1x * Ux - f2x * Uxx);
                  rec2 = f0y * u0 - (f1y * Vy - f2y * Vyy);
                } else {
                  rhs = fma(a, xsup ? (T)0 : Ux, fma(bb, ysup ? (T)0 : Vy, rhs));
                  if (src_bnd) rhs += 4 * (a * xa0 + bb * ya0);
                  const int bi = (xbnd ? 1 : (xsup ? 2 : 0)) + 3 * (ybnd ? 1 : (ysup ? 2 : 0));
                  const T inv = TAB ? tload(cf + kA[k] + bi)
                                    : rcp(2 * st + a * (T)(xbnd ? 4 : (xsup ? 2 : 3)) +
                                          bb * (T)(ybnd ? 4 : (ysup ? 2 : 3)));
                  u0 = rhs * inv;
                  rec1 = (xbnd ? (T)1 : (xsup ? (T)0 : (T)0.5)) * (u0 - Ux);
                  rec2 = (ybnd ? (T)1 : (ysup ? (T)0 : (T)0.5)) * (u0 - Vy);
                }
                if (src_bnd) { rec1 -= xa0; rec2 -= ya0; }
                // direction-dependent part of L(u; b_r): u1 = A1 + rec1, u2 = A2 + rec2, inflow traces U, V
                //   r=1: 2a (U0 - u0) + (2a + 2/3 b) rec1 - 2/3 b V1   (2/3 sigma_t h rec1: epilogue)
                //   r=2: 2b (V0 - u0) + (2b + 2/3 a) rec2 - 2/3 a U1
                //   r=3: 2/3 a (U1 - rec2) + 2/3 b (V1 - rec1)
                if constexpr (Q1R) {
                  // Q1-type: u3 = A3 + rec3 with the xi eta coefficient rec3 = (h/2)^2 delta_xy, the upwind
                  // y-difference of the x-slopes: (rec1 - rec1 of the cell below) / 2 inside, rec1 - a1 on the
                  // y-inflow row (a1 the along-face coefficient of the inflow data there, local orientation).  It
                  // adds 2/3 b rec3, 2/3 a rec3 and 2/3 (a + b) rec3 to rows 1, 2, 3 (2/9 sigma_t h rec3: epilogue)
                  // and rides on the traces' slopes (U1, V1); row 0 does not see it
                  const T rec3 = ybnd ? rec1 - ya1 : (T)0.5 * (rec1 - yin[3]);
                  if (use_corr) {
                    acc[0] += wl * u0 * (T)A.corr[(size_t)cA[k] * plane + rslot];
                  } else {
                    acc[0] = fma(wl, u0, acc[0]);
                    acc[1] = fma(nWxb[k], V1 - rec3, fma(Dx[k], rec1, fma(Wx[k], U0 - u0, acc[1])));
                    acc[2] = fma(nWya[k], U1 - rec3, fma(Dy[k], rec2, fma(Wy[k], V0 - u0, acc[2])));
                    acc[3] = fma(W3b[k], V1 - rec1 + rec3, fma(W3a[k], U1 - rec2 + rec3, acc[3]));
                  }
                  acc[4] = fma(wx[k], rec1, acc[4]);
                  acc[5] = fma(wy[k], rec2, acc[5]);
                  acc[6] = fma(wxy[k], rec3, acc[6]);
                  xs[k][0] = u0 + A1 + rec1; xs[k][1] = A23 + rec2 + rec3; xs[k][2] = u0;
                  ys[k][0] = u0 + A2 + rec2; ys[k][1] = A13 + rec1 + rec3; ys[k][2] = u0; ys[k][3] = rec1;
                } else {
                  if (use_corr) {
                    acc[0] += wl * u0 * (T)A.corr[(size_t)cA[k] * plane + rslot];
                  } else {
                    acc[0] = fma(wl, u0, acc[0]);
                    acc[1] = fma(nWxb[k], V1, fma(Dx[k], rec1, fma(Wx[k], U0 - u0, acc[1])));
                    acc[2] = fma(nWya[k], U1, fma(Dy[k], rec2, fma(Wy[k], V0 - u0, acc[2])));
                    acc[3] = fma(W3b[k], V1 - rec1, fma(W3a[k], U1 - rec2, acc[3]));
                  }
                  acc[4] = fma(wx[k], rec1, acc[4]);
                  acc[5] = fma(wy[k], rec2, acc[5]);
                  if constexpr (VAR == 3) { xs[k][3] = Ux; ys[k][3] = Vy; }
                  xs[k][0] = u0 + A1 + rec1; xs[k][1] = A23 + rec2; xs[k][2] = u0;
                  ys[k][0] = u0 + A2 + rec2; ys[k][1] = A13 + rec1; ys[k][2] = u0;
                }
                if (LSTORE || (!LEAN && A.psi)) store_psi0<T>(A.psi, (size_t)uA[k] * plane + pslot, u0, A.psi_bf16);
              }
              if (lane == 31 && has_above) {
                T *yp = A.ytr + (((size_t)ang[k] * A.g.strips + strip) * ni + x) * kTraceStride;
#pragma unroll
                for (int c = 0; c < NS; ++c) st_trace(yp + c, ys[k][c]);
              }
            }
          }
        }
        if (VAR == 1 && act) {
          if (nA > 0 && !use_corr) {
            // slope-trace terms, the same for every direction: -2/3 b V1 (r=1), -2/3 a U1 (r=2),
            // 2/3 (a U1 + b V1) (r=3), U1 = the left cell's A2 + A3, V1 = the lower cell's A1 + A3
            acc[1] += nGb * yl1_in;
            acc[2] += nGa * xl1;
            acc[3] += G3a * xl1 + G3b * yl1_in;
          }
          xl1 = A23;
          yl1 = A13;
        }
        store_nr<T, NR>(red + ((size_t)((b * C + s) * W + warp) * 32 + lane) * NR, acc);
      }
    }

    // ---- end of chunk: one barrier, then a fixed-order sum over the warps
    cp_async_wait_all();
    __syncthreads();
    if (s_abort) return;
    for (int it = threadIdx.x; it < C * 32; it += blockDim.x) {
      const int s = it >> 5, l = it & 31;
      const int t = t0 + s, x = t - l, r = strip * 32 + l;
      if (t >= nsteps || r >= nj || x < 0 || x >= ni) continue;
      const int ii = sx > 0 ? x : ni - 1 - x, jj = sy > 0 ? r : nj - 1 - r;
      const size_t K = (size_t)jj * ni + ii;
      T sum[NR];
      load_nr<T, NR>(sum, red + ((size_t)((b * C + s) * W) * 32 + l) * NR);   // warp 0, then the others in order
      for (int ww = 1; ww < Wact; ++ww) {
        add_nr<T, NR>(sum, red + ((size_t)((b * C + s) * W + ww) * 32 + l) * NR);
      }
      T *dst = A.part + ((size_t)pq * nx + K) * NR;
      store_nr<T, NR>(dst, sum);
    }
  }
}

// Quadrature moments used by the epilogue: [sum w, sum w |Omega_x|, sum w |Omega_y|, sum w Omega_x, sum w Omega_y]
// over all directions, summed in index order.
__global__ void quad_moments_kernel(int nang, const double *__restrict__ ox, const double *__restrict__ oy,
                                    const double *__restrict__ w, double *__restrict__ qm) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double m[5] = {0, 0, 0, 0, 0};
  for (int l = 0; l < nang; ++l) {
    m[0] += w[l];
    m[1] += w[l] * fabs(ox[l]);
    m[2] += w[l] * fabs(oy[l]);
    m[3] += w[l] * ox[l];
    m[4] += w[l] * oy[l];
  }
  for (int r = 0; r < 5; ++r) qm[r] = m[r];
}

// y = K X - source * b from the partial reductions, one thread per cell.
//   STD : y = X - sum_p part_p                       (K = I - P L^-1 M; b = P L^-1 Q)
//   LM/RLM: y0 = X0 - P0 psi0
//           y_r = (sigma_s/eps) h^2 D_r (S_r - source P1r_alpha_r - X_r) - (h/2) T_r + source SigmaQ1_r
// where T_r = sum_l w_l L_l(u_l; b_r) over the full trial functions u_l = psi0_l + (R psi0)_l - X1 and S = P1 R
// psi0.  For the homogeneous sweep this equals the second block row B11 X1 - (Sigma Ltilde10 + B11 P1 R) psi0
// of the reduced operator, because Sigma L11 Sigma^T = B11 + Sigma M1 (eq-lmdg-psi1).  The partials hold the
// direction-dependent part of T_r; the part through the cell's own isotropic slopes A_r = -(X_r + source
// P1r_alpha_r) is added here with the quadrature moments qm (s = sigma_t h, c = 2/3):
//   T_1 += (2 Ma + c Mb + c s Mw) A_1 + c MOy A_3 [+ c s sum w sx rec_1]
//   T_2 += (2 Mb + c Ma + c s Mw) A_2 + c MOx A_3 [+ c s sum w sy rec_2]
//   T_3 += -c MOy A_1 - c MOx A_2 + (c (Ma + Mb) + 2/9 s Mw) A_3
template <typename T, int VAR>
__global__ void epilogue_kernel(int nx, int P, double h, const T *__restrict__ part,
                                const double *__restrict__ X, const double *__restrict__ sse,
                                const double *__restrict__ sigt, const double *__restrict__ qm,
                                const double *__restrict__ p1ra, const double *__restrict__ sq1, int source,
                                double *__restrict__ y) {
  constexpr int NR = nr_of(VAR);
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nx) return;
  // the partials in index order, four quadrant-groups' loads in flight at a time.  FP32 partials are summed in
  // FP32 with Neumaier's compensation and converted once (sum + compensation in FP64): as accurate as an FP64
  // sum, without a float-to-double conversion and an FP64 addition per partial (FP64 is the scarce pipe).
  // Float-float partials are summed in float-float and converted once.
  double s[NR];
  T hs[NR], hc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { hs[r] = 0; hc[r] = 0; }
  auto add = [&](const T *v) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if constexpr (sizeof(T) == 4) {
        const T t = hs[r] + v[r];
        hc[r] += (fabsf(hs[r]) >= fabsf(v[r])) ? ((hs[r] - t) + v[r]) : ((v[r] - t) + hs[r]);
        hs[r] = t;
      } else {
        hs[r] += v[r];
      }
    }
  };
  int p = 0;
  for (; p + 4 <= P; p += 4) {
    T v[4][NR];
#pragma unroll
    for (int i = 0; i < 4; ++i) load_nr<T, NR>(v[i], part + ((size_t)(p + i) * nx + K) * NR);
#pragma unroll
    for (int i = 0; i < 4; ++i) add(v[i]);
  }
  for (; p < P; ++p) {
    T v[NR];
    load_nr<T, NR>(v, part + ((size_t)p * nx + K) * NR);
    add(v);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) s[r] = sizeof(T) == 4 ? (double)hs[r] + (double)hc[r] : (double)hs[r];
  const double2 xa = *reinterpret_cast<const double2 *>(X + 4 * (size_t)K);
  const double2 xb = *reinterpret_cast<const double2 *>(X + 4 * (size_t)K + 2);
  double o0, o1, o2, o3;
  if constexpr (VAR == 0) {
    o0 = xa.x - s[0]; o1 = xa.y - s[1]; o2 = xb.x - s[2]; o3 = xb.y - s[3];
  } else if constexpr (VAR == kP0) {
    o0 = xa.x - s[0]; o1 = xa.y; o2 = xb.x; o3 = xb.y;   // P0-DG: the slope entries are carried by the identity
  } else {
    const double m = sse[K] * h * h;
    const double c = 2.0 / 3.0, sh = sigt[K] * h;
    const double Mw = qm[0], Ma = qm[1], Mb = qm[2], MOx = qm[3], MOy = qm[4];
    double S1 = 0, S2 = 0, S3 = 0, p1 = 0, p2 = 0, p3 = 0;
    if constexpr (VAR >= 2) {
      S1 = s[4]; S2 = s[5];
      if constexpr (VAR == kRlmQ1) S3 = s[6];   // P1 R psi0 of the xi eta term (Q1-type reconstruction)
      if (source && p1ra) {
        p1 = p1ra[3 * (size_t)K]; p2 = p1ra[3 * (size_t)K + 1]; S1 -= p1; S2 -= p2;
        if constexpr (VAR == kRlmQ1) { p3 = p1ra[3 * (size_t)K + 2]; S3 -= p3; }
      }
    }
    const double A1 = -(xa.y + p1), A2 = -(xb.x + p2), A3 = -(xb.y + p3);
    double T1 = s[1] + (2 * Ma + c * Mb + c * sh * Mw) * A1 + c * MOy * A3;
    double T2 = s[2] + (2 * Mb + c * Ma + c * sh * Mw) * A2 + c * MOx * A3;
    double T3 = s[3] - c * MOy * A1 - c * MOx * A2 + (c * (Ma + Mb) + (2.0 / 9.0) * sh * Mw) * A3;
    if constexpr (VAR >= 2) { T1 += c * sh * s[4]; T2 += c * sh * s[5]; }
    if constexpr (VAR == kRlmQ1) T3 += (2.0 / 9.0) * sh * s[6];
    o0 = xa.x - s[0];
    o1 = m * (1.0 / 3.0) * (S1 - xa.y) - 0.5 * h * T1;
    o2 = m * (1.0 / 3.0) * (S2 - xb.x) - 0.5 * h * T2;
    o3 = m * (1.0 / 9.0) * (S3 - xb.y) - 0.5 * h * T3;
    if (source && sq1) { o1 += sq1[3 * (size_t)K]; o2 += sq1[3 * (size_t)K + 1]; o3 += sq1[3 * (size_t)K + 2]; }
  }
  *reinterpret_cast<double2 *>(y + 4 * (size_t)K) = make_double2(o0, o1);
  *reinterpret_cast<double2 *>(y + 4 * (size_t)K + 2) = make_double2(o2, o3);
}

template <typename T, int VAR, int APW, bool TAB, bool LEAN, bool LSTORE>
static const void *kernel_ptr() {
  return reinterpret_cast<const void *>(&sweep_kernel<T, VAR, APW, TAB, LEAN, LSTORE>);
}

template <typename T, int VAR, bool TAB, bool LEAN, bool LSTORE>
static const void *kernel_for(int apw) {
  // float-float sweeps and the lean storing instances: one or two directions per warp (choose_geom's FP32 and
  // float-float shapes)
  if constexpr (is_f2<T>::value || LSTORE) {
    return apw == 1 ? kernel_ptr<T, VAR, 1, TAB, LEAN, LSTORE>() : kernel_ptr<T, VAR, 2, TAB, LEAN, LSTORE>();
  } else {
    switch (apw) {
      case 1: return kernel_ptr<T, VAR, 1, TAB, LEAN, false>();
      case 2: return kernel_ptr<T, VAR, 2, TAB, LEAN, false>();
      case 3: return kernel_ptr<T, VAR, 3, TAB, LEAN, false>();
      default: return kernel_ptr<T, VAR, 4, TAB, LEAN, false>();
    }
  }
}

template <typename T, bool TAB, bool LEAN, bool LSTORE = false>
static const void *kernel_for_variant(int variant, int apw) {
  switch (variant) {
    case LMDG_STD: return kernel_for<T, 0, TAB, LEAN, LSTORE>(apw);
    case LMDG_LM: return kernel_for<T, 1, TAB, LEAN, LSTORE>(apw);
    case LMDG_RLM: return kernel_for<T, 2, TAB, LEAN, LSTORE>(apw);
    case kRlmStar: return kernel_for<T, 3, TAB, LEAN, LSTORE>(apw);
    case kRlmQ1: return kernel_for<T, kRlmQ1, TAB, LEAN, LSTORE>(apw);
    default: return kernel_for<T, kP0, TAB, LEAN, LSTORE>(apw);
  }
}

// coefficient tables exist for the FP64 and float-float sweeps; lean instances for FP32 and float-float, lean
// storing ones for FP32 with one or two directions per warp
template <typename T>
static const void *sweep_kernel_ptr(int variant, int apw, bool tab, bool lean, bool lstore = false) {
  constexpr bool kLean = !std::is_same<T, double>::value;
  if constexpr (std::is_same<T, float>::value) {
    if (lstore && apw <= 2) return kernel_for_variant<T, false, true, true>(variant, apw);
  }
  (void)lstore;
  if constexpr (sizeof(T) == 8) {
    if (tab) {
      if constexpr (kLean) {
        if (lean) return kernel_for_variant<T, true, true>(variant, apw);
      }
      return kernel_for_variant<T, true, false>(variant, apw);
    }
  }
  if constexpr (kLean) {
    if (lean) return kernel_for_variant<T, false, true>(variant, apw);
  }
  (void)tab;
  (void)lean;
  return kernel_for_variant<T, false, false>(variant, apw);
}

template <typename T>
int sweep_blocks_per_sm(int variant, int warps, int apw) {
  const void *k = sweep_kernel_ptr<T>(variant, apw, false, false);
  const size_t smem = sweep_smem_bytes<T>(variant, warps, apw);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess) return 0;
  return nb;
}

template <typename T>
cudaError_t launch_sweep(int variant, const SweepArgs<T> &a, cudaStream_t s) {
  // per-cell inputs in the sweep's precision
  {
    const int bs = 256, gs = (a.nx + bs - 1) / bs;
    add_launches(1);
    T *src = const_cast<T *>(a.cellsrc), *sh = const_cast<T *>(a.cellsh);
    const int qiso = a.q_per_angle ? 0 : 1;
    switch (variant) {
      case LMDG_STD:
        prep_kernel<T, 0><<<gs, bs, 0, s>>>(a.nx, a.h, a.eps, a.X, a.pd.sse, a.pd.sigt, a.pd.q, a.p1ra, a.source,
                                            qiso, src, sh, a.coef ? a.mat : nullptr);
        break;
      case LMDG_LM:
        prep_kernel<T, 1><<<gs, bs, 0, s>>>(a.nx, a.h, a.eps, a.X, a.pd.sse, a.pd.sigt, a.pd.q, a.p1ra, a.source,
                                            qiso, src, sh, a.coef ? a.mat : nullptr);
        break;
      case kP0:
        prep_kernel<T, kP0><<<gs, bs, 0, s>>>(a.nx, a.h, a.eps, a.X, a.pd.sse, a.pd.sigt, a.pd.q, a.p1ra,
                                              a.source, qiso, src, sh, a.coef ? a.mat : nullptr);
        break;
      default:
        prep_kernel<T, 2><<<gs, bs, 0, s>>>(a.nx, a.h, a.eps, a.X, a.pd.sse, a.pd.sigt, a.pd.q, a.p1ra, a.source,
                                            qiso, src, sh, a.coef ? a.mat : nullptr);
        break;
    }
  }
  cudaError_t e = cudaMemsetAsync(a.ctrl, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  // lean: nothing a lean instance leaves out is needed -- a source sweep without inflow data or angle-dependent
  // source (its source enters through prep_kernel's cell data) runs the same per-step code as a homogeneous one
  const bool plain = !(a.source && (a.pd.alpha != nullptr || a.q_per_angle)) && a.corr == nullptr;
  const bool lean = plain && a.psi == nullptr;
  const void *k = sweep_kernel_ptr<T>(variant, a.g.apw, a.coef != nullptr, lean, plain && a.psi != nullptr);
  const size_t smem = sweep_smem_bytes<T>(variant, a.g.warps, a.g.apw);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  SweepArgs<T> args = a;
  void *params[] = {&args};
  add_launches(1);
  if (a.npq < 1 || a.pq0 < 0 || a.pq0 + a.npq > 4 * a.g.groups) return cudaErrorInvalidValue;
  e = cudaLaunchKernel(k, dim3(a.g.strips * a.npq), dim3(a.g.warps * 32), params, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t quad_moments(int nang, const double *ox, const double *oy, const double *w, double *qm, cudaStream_t s) {
  add_launches(1);
  quad_moments_kernel<<<1, 32, 0, s>>>(nang, ox, oy, w, qm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_epilogue(int variant, int nx, int P, double h, const T *part, const double *X,
                            const double *sse, const double *sigt, const double *qm, const double *p1ra,
                            const double *sq1, int source, double *y, cudaStream_t s) {
  const int bs = 256, gs = (nx + bs - 1) / bs;
  add_launches(1);
  switch (variant) {
    case LMDG_STD:
      epilogue_kernel<T, 0><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, sigt, qm, p1ra, sq1, source, y);
      break;
    case LMDG_LM:
      epilogue_kernel<T, 1><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, sigt, qm, p1ra, sq1, source, y);
      break;
    case kP0:
      epilogue_kernel<T, kP0><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, sigt, qm, p1ra, sq1, source, y);
      break;
    case kRlmQ1:
      epilogue_kernel<T, kRlmQ1><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, sigt, qm, p1ra, sq1, source, y);
      break;
    default:
      epilogue_kernel<T, 2><<<gs, bs, 0, s>>>(nx, P, h, part, X, sse, sigt, qm, p1ra, sq1, source, y);
      break;
  }
  return cudaGetLastError();
}

__global__ void to_f2_kernel(size_t n, const double *__restrict__ x, f2 *__restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2(x[i]);
}

cudaError_t convert_to_f2(const double *x, f2 *y, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  add_launches(1);
  to_f2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

template size_t sweep_smem_bytes<double>(int, int, int);
template size_t sweep_smem_bytes<float>(int, int, int);
template size_t sweep_smem_bytes<f2>(int, int, int);
template int sweep_blocks_per_sm<double>(int, int, int);
template int sweep_blocks_per_sm<float>(int, int, int);
template int sweep_blocks_per_sm<f2>(int, int, int);
template cudaError_t launch_sweep<double>(int, const SweepArgs<double> &, cudaStream_t);
template cudaError_t launch_sweep<float>(int, const SweepArgs<float> &, cudaStream_t);
template cudaError_t launch_sweep<f2>(int, const SweepArgs<f2> &, cudaStream_t);
template cudaError_t launch_epilogue<double>(int, int, int, double, const double *, const double *, const double *,
                                             const double *, const double *, const double *, const double *, int,
                                             double *, cudaStream_t);
template cudaError_t launch_epilogue<float>(int, int, int, double, const float *, const double *, const double *,
                                            const double *, const double *, const double *, const double *, int,
                                            double *, cudaStream_t);
template cudaError_t launch_epilogue<f2>(int, int, int, double, const f2 *, const double *, const double *,
                                         const double *, const double *, const double *, const double *, int,
                                         double *, cudaStream_t);

}  // namespace lmdg
