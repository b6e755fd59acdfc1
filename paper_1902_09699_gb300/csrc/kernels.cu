// PARSDMM iteration kernels for sm_103a (internal to libsip.so).
//
// One iteration of Algorithm PARSDMM (Eq. SDMM_adaptive) is the launch
// sequence
//   k_rhs        b = sum_i A_i^T(rho_i y_i + v_i) (+ m, direct form);
//                r = b - C x                      (x-update right-hand side)
//   k_cg_dir     p = r + beta p; q = C p; p.q     } x n_cg   (warm-started CG,
//   k_cg_upd     x += alpha p; r -= alpha q; r.r  }           Sec. "Solving the
//                                                             linear system ...")
//   k_setpass    every block: s_i = A_i x, xbar_i, w_i, point-wise prox and
//                dual update; w_i stored for l1 / l2 / card sets; feasibility
//                (Eq. feas_stop), evolution (Eq. obj_stop) and adapt-rho-gamma
//                inner products
//   k_select     radix-select passes for l1 thresholds and top-k
//   k_ties       card tie ranks (only when the k-th value is tied)
//   k_final      l1 / l2 / card prox from the stored w_i and the dual update
//   k_tail       per instance: r_feas, r_evol, stopping rule, Algorithm
//                adapt-rho-gamma, new stencil coefficients of C, k += 1
// All scalars live on the device; reductions are binary64 across threads and
// finish in the last CTA to arrive ("last tile"), so no launch waits on the
// host.
//
// Work decomposition: every launch walks a list of work items; one CTA owns
// one item (a contiguous run of grid points / rows of one instance, segment,
// block or selection job) and walks it in steps of PT rows per thread
// (PerThread<T>).  Inside a step every thread first issues all of its
// global loads and only then computes, so the memory system sees many
// independent requests per thread.  Per-CTA partial sums are merged with one
// set of binary64 atomics per CTA.
#include <cstdint>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "sip_dev.cuh"
#include "sip_kernels.h"

namespace sip {

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ double ldv(const double *p) { return *(const volatile double *)p; }

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums NQ values over the CTA in their own type; thread 0 gets the totals.
// (Binary64 arithmetic issues at a small fraction of the binary32 rate on
// this part, so binary32 data is summed in binary32 within a CTA.)
template <int NQ, typename A>
__device__ __forceinline__ void block_sum(A (&v)[NQ]) {
  __shared__ A sm[NQ][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    A t = warp_sum(v[q]);
    if (lane == 0) sm[q][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      A t = lane < kThreads / 32 ? sm[q][lane] : A(0);
      v[q] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Exact sum of two binary32 numbers as an unevaluated pair s + e (Knuth's
// TwoSum: s = fl(a + b), e = a + b - s exactly, for any order of a, b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Totals of NQ per-tile partial arrays p[q][0..nt), formed by all threads of
// the CTA in a fixed order (thread-strided sums, a butterfly in each warp
// whose two partners add the same operands, then the warps in order), so
// every CTA that reads the same partials gets the same bits.  Binary32
// partials are added in double-binary32 arithmetic (hi + lo, the rounding
// error of each addition kept by TwoSum), binary64 partials in binary64.
// Thread 0 gets the totals (binary32 partials: in binary32, or as hi + lo in
// binary64); the call contains __syncthreads.
constexpr int kGatherBatch = 2;  // loads in flight per thread and quantity

__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2) {
  float sum, err;
  two_sum(hi, h2, sum, err);
  hi = sum;
  lo = (lo + l2) + err;
}

// This thread's entries of the first batch (entries threadIdx.x + u kThreads).
template <int NQ>
__device__ __forceinline__ void gather_first(const float *const (&p)[NQ], int nt, float (&v)[NQ][kGatherBatch]) {
#pragma unroll
  for (int u = 0; u < kGatherBatch; ++u) {
    const int i = u * kThreads + threadIdx.x;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q][u] = i < nt ? __ldcg(p[q] + i) : 0.f;
  }
}

// pre: the first batch, already loaded by gather_first (or null)
template <int NQ, typename O>
__device__ __forceinline__ void cta_gather(const float *const (&p)[NQ], int nt, O (&out)[NQ],
                                           const float (*pre)[kGatherBatch] = nullptr) {
  constexpr int NW = kThreads / 32;
  __shared__ float sh[NQ][NW], sl[NQ][NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float hi[NQ], lo[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) hi[q] = lo[q] = 0.f;
  for (int i0 = 0; i0 < nt; i0 += kThreads * kGatherBatch) {
    float v[NQ][kGatherBatch];
    if (pre && i0 == 0) {
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u)
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q][u] = pre[q][u];
    } else {
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u) {
        const int i = i0 + u * kThreads + threadIdx.x;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q][u] = i < nt ? __ldcg(p[q] + i) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) df_add(hi[q], lo[q], v[q][u], 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      df_add(hi[q], lo[q], __shfl_xor_sync(0xffffffffu, hi[q], o), __shfl_xor_sync(0xffffffffu, lo[q], o));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      sh[q][wid] = hi[q];
      sl[q][wid] = lo[q];
    }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float H = sh[q][0], L = sl[q][0];
      for (int w = 1; w < NW; ++w) df_add(H, L, sh[q][w], sl[q][w]);
      out[q] = sizeof(O) == 4 ? (O)(H + L) : (O)H + (O)L;
    }
}
template <int NQ>
__device__ __forceinline__ void cta_gather(const double *const (&p)[NQ], int nt, double (&out)[NQ]) {
  constexpr int NW = kThreads / 32;
  __shared__ double sh[NQ][NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double t[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) t[q] = 0.0;
  for (int i0 = 0; i0 < nt; i0 += kThreads * kGatherBatch) {
    double v[NQ][kGatherBatch];
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) {
      const int i = i0 + u * kThreads + threadIdx.x;
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q][u] = i < nt ? __ldcg(p[q] + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) t[q] += v[q][u];
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double w = warp_sum(t[q]);
    if (lane == 0) sh[q][wid] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double tot = sh[q][0];
      for (int w = 1; w < NW; ++w) tot += sh[q][w];
      out[q] = tot;
    }
}

// Called by thread 0 after its atomics: true in the last CTA of a group.
__device__ __forceinline__ bool arrive_last(uint32_t *counter, uint32_t n) {
  __threadfence();
  uint32_t prev = atomicAdd(counter, 1u);
  if (prev == n - 1) {
    atomicExch(counter, 0u);
    __threadfence();
    return true;
  }
  return false;
}

// Partial sums within a CTA: binary32 for binary32 storage, binary64
// otherwise; sums across CTAs are binary64 (or double-binary32, see
// cta_gather).
template <typename T> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float; };

// Rows per thread per step: 4 in binary32, 2 in binary64 (register budget).
template <typename T> struct PerThread { static constexpr int value = 2; };
template <> struct PerThread<float> { static constexpr int value = 4; };
#define SIP_STEP_CONSTANTS                               \
  constexpr int PT = PerThread<T>::value;                \
  constexpr int SUB = kThreads * PT;                     \
  static_assert(kTile % SUB == 0, "step must divide kTile")

__device__ __forceinline__ bool adapt_iter(const InstDev &in, int k) {
  return in.adapt != 0 && in.rho_sched == nullptr &&
         (k % in.adapt_every) == (1 % in.adapt_every);
}
__device__ __forceinline__ bool check_iter(const InstDev &in, int k) { return (k % in.check_every) == 0; }

// Per-iteration scalars in the storage type.  The binary64 values are
// authoritative; binary32 kernels read the binary32 copies the tails write
// next to them, so no hot loop converts between precisions.
enum BlkField : int { BF_RHO = 0, BF_IRHO, BF_GAMMA, BF_OMG, BF_INV1P, BF_L2SCALE };
template <typename T> struct SV;
template <> struct SV<double> {
  static __device__ __forceinline__ double c(const InstScal &s, int i) {
    return i == 0 ? s.c0 : i == 1 ? s.cz : i == 2 ? s.cx : s.cy;
  }
  static __device__ __forceinline__ double blk(const InstScal &s, int b, int f) {
    switch (f) {
      case BF_RHO: return s.rho[b];
      case BF_IRHO: return s.irho[b];
      case BF_GAMMA: return s.gamma[b];
      case BF_OMG: return 1.0 - s.gamma[b];
      case BF_INV1P: return s.inv1p[b];
      default: return s.l2scale[b];
    }
  }
  static __device__ __forceinline__ double ih(const InstDev &in, int axis) {
    return axis == 0 ? in.ihz : axis == 1 ? in.ihx : in.ihy;
  }
  static __device__ __forceinline__ double theta(const JobScal &j) { return j.theta; }
};
template <> struct SV<float> {
  static __device__ __forceinline__ float c(const InstScal &s, int i) { return s.cf[i]; }
  static __device__ __forceinline__ float blk(const InstScal &s, int b, int f) { return s.bf[b][f]; }
  static __device__ __forceinline__ float ih(const InstDev &in, int axis) {
    return axis == 0 ? in.ihzf : axis == 1 ? in.ihxf : in.ihyf;
  }
  static __device__ __forceinline__ float theta(const JobScal &j) { return j.thetaf; }
};

// binary32 copies of the block scalars after rho / gamma / l2 scale changed
__device__ __forceinline__ void store_block_f32(InstScal &sc, int b) {
  sc.bf[b][BF_RHO] = (float)sc.rho[b];
  sc.bf[b][BF_IRHO] = (float)sc.irho[b];
  sc.bf[b][BF_GAMMA] = (float)sc.gamma[b];
  sc.bf[b][BF_OMG] = (float)(1.0 - sc.gamma[b]);
  sc.bf[b][BF_INV1P] = (float)sc.inv1p[b];
  sc.bf[b][BF_L2SCALE] = (float)sc.l2scale[b];
}
__device__ __forceinline__ void store_coef_f32(InstScal &sc) {
  sc.cf[0] = (float)sc.c0;
  sc.cf[1] = (float)sc.cz;
  sc.cf[2] = (float)sc.cx;
  sc.cf[3] = (float)sc.cy;
}

// Grid position of a linear index g (z fastest).
struct GridPos {
  int32_t iz, ix, iy;
  int64_t t;  // ix + nx*iy
};
template <typename D>
__device__ __forceinline__ GridPos grid_pos(const D &in, int64_t g) {
  GridPos p;
  const uint32_t gg = (uint32_t)g;
  const uint32_t t = fdiv(gg, in.fz);
  p.iz = (int32_t)(gg - t * (uint32_t)in.nz);
  p.t = t;
  const uint32_t iy = fdiv(t, in.fx);
  p.iy = (int32_t)iy;
  p.ix = (int32_t)(t - iy * (uint32_t)in.nx);
  return p;
}

// Grid index of the base sample of a row of a difference segment and the
// offset of its partner sample (Eq. FD_mat: row = (x[g + off] - x[g]) / h).
__device__ __forceinline__ int64_t seg_base(const InstDev &in, int kind, int64_t row, int64_t &off) {
  switch (kind) {
    case SEG_DZ: {
      const uint32_t t = fdiv((uint32_t)row, in.fzm);  // ix + nx*iy
      off = 1;
      return row + t;
    }
    case SEG_DX: {
      const uint32_t t = fdiv((uint32_t)row, in.fz);   // ix + (nx-1)*iy
      const uint32_t iy = fdiv(t, in.fxm);
      off = in.nz;
      return row + (int64_t)in.nz * iy;
    }
    case SEG_DY:
      off = (int64_t)in.nz * in.nx;
      return row;
    default:
      off = 0;
      return row;
  }
}

template <typename T>
__device__ __forceinline__ T seg_ih(const InstDev &in, int kind) {
  return kind == SEG_DZ ? SV<T>::ih(in, 0) : kind == SEG_DX ? SV<T>::ih(in, 1) : kind == SEG_DY ? SV<T>::ih(in, 2) : T(1);
}

// Blurring forward operator F of a data-fit block (sip_op SIP_OP_BLUR):
// (F v)[g] = sum_{|t| <= R} k_|t| v[g + t st] along the blur axis, samples
// outside the grid taken as 0.  F is symmetric, so F^T = F.
template <typename D>
__device__ __forceinline__ int blur_pos(const D &in, int64_t g) {
  if (in.bl_axis == 0) return (int)((uint32_t)g - (uint32_t)in.nz * fdiv((uint32_t)g, in.fz));
  const uint32_t t = fdiv((uint32_t)g, in.fz);  // ix + nx*iy
  if (in.bl_axis == 1) return (int)(t - (uint32_t)in.nx * fdiv(t, in.fx));
  return (int)fdiv(t, in.fx);
}
template <typename T, typename D, typename V>
__device__ __forceinline__ T blur_fwd(const D &in, int64_t g, V v) {
  const T *__restrict__ k = (const T *)in.bl_w;
  const int R = in.bl_R, n = in.bl_n, i = blur_pos(in, g);
  const int64_t st = in.bl_st;
  T s = k[0] * v(g);
  for (int t = 1; t <= R; ++t) {
    const T a = i - t >= 0 ? v(g - t * st) : T(0);
    const T b = i + t < n ? v(g + t * st) : T(0);
    s += k[t] * (a + b);
  }
  return s;
}
// s = A x for one row of a segment (used by the single-step entry points and
// the norm kernel; the loop kernels inline the same arithmetic).
template <typename T>
__device__ __forceinline__ T seg_forward(const InstDev &in, int kind, const T *__restrict__ x, int64_t row,
                                         int64_t &g) {
  int64_t off;
  g = seg_base(in, kind, row, off);
  if (kind == SEG_I || kind == SEG_RING) return x[g];
  if (kind == SEG_BLUR) return blur_fwd<T>(in, g, [&](int64_t q) { return x[q]; });
  return (x[g + off] - x[g]) * seg_ih<T>(in, kind);
}

// (A^T u)[g] for one segment, where u(row) is supplied by a functor over the
// segment's rows: columns of the bidiagonal difference matrix (Eq. FD_mat).
template <typename T, typename U>
__device__ __forceinline__ T seg_adjoint(const InstDev &in, int kind, const GridPos &p, int64_t g, U u) {
  switch (kind) {
    case SEG_DZ: {
      const int64_t r = g - p.t;  // iz + (nz-1)*t
      T a = p.iz >= 1 ? u(r - 1) : T(0);
      T b = p.iz <= in.nz - 2 ? u(r) : T(0);
      return (a - b) * SV<T>::ih(in, 0);
    }
    case SEG_DX: {
      const int64_t r = g - (int64_t)in.nz * p.iy;  // iz + nz*(ix + (nx-1)*iy)
      T a = p.ix >= 1 ? u(r - in.nz) : T(0);
      T b = p.ix <= in.nx - 2 ? u(r) : T(0);
      return (a - b) * SV<T>::ih(in, 1);
    }
    case SEG_DY: {
      const int64_t s = (int64_t)in.nz * in.nx;
      T a = p.iy >= 1 ? u(g - s) : T(0);
      T b = p.iy <= in.ny - 2 ? u(g) : T(0);
      return (a - b) * SV<T>::ih(in, 2);
    }
    default:
      return u(g);
  }
}

// Coefficients of C = c0 I + cz D_z^T D_z + cx D_x^T D_x + cy D_y^T D_y
// (Eq. sys_mat) in the storage type; D^T D along an axis is the Neumann
// second difference.
template <typename T>
struct CSys {
  T c0, cz, cx, cy;
  __device__ __forceinline__ void load(const InstScal &sc) {
    c0 = SV<T>::c(sc, 0);
    cz = SV<T>::c(sc, 1);
    cx = SV<T>::c(sc, 2);
    cy = SV<T>::c(sc, 3);
  }
};

// Values of a vector v (v(i) = functor) at the 7-point stencil of g; the
// neighbours that fall outside the grid are not read.
template <typename T>
struct Nbr {
  T c, zm, zp, xm, xp, ym, yp;
};
template <typename T, typename V, typename D>
__device__ __forceinline__ void load_nbr(const D &in, const GridPos &p, int64_t g, V v, Nbr<T> &o) {
  const int64_t sxy = (int64_t)in.nz * in.nx;
  o.c = v(g);
  o.zm = p.iz > 0 ? v(g - 1) : o.c;
  o.zp = p.iz < in.nz - 1 ? v(g + 1) : o.c;
  o.xm = p.ix > 0 ? v(g - in.nz) : o.c;
  o.xp = p.ix < in.nx - 1 ? v(g + in.nz) : o.c;
  o.ym = p.iy > 0 ? v(g - sxy) : o.c;
  o.yp = p.iy < in.ny - 1 ? v(g + sxy) : o.c;
}
// A missing neighbour was loaded as the centre value, so its difference is 0:
// exactly the Neumann (no boundary row) second difference of Eq. FD_mat.
template <typename T>
__device__ __forceinline__ T apply_c(const CSys<T> &C, const Nbr<T> &n) {
  const T lz = (n.c - n.zm) + (n.c - n.zp);
  const T lx = (n.c - n.xm) + (n.c - n.xp);
  const T ly = (n.c - n.ym) + (n.c - n.yp);
  return C.c0 * n.c + C.cz * lz + C.cx * lx + C.cy * ly;
}

template <typename T, typename V>
__device__ __forceinline__ T csys(const InstDev &in, const InstScal &sc, const GridPos &p, int64_t g, V v) {
  CSys<T> C;
  C.load(sc);
  Nbr<T> n;
  load_nbr<T>(in, p, g, v, n);
  return apply_c(C, n);
}


// Launch-time stamps of the timing runs: thread 0 of every CTA folds the
// global nanosecond timer at its start into ts[0] (minimum) and the
// complement of the timer at its end into ts[1] (minimum, i.e. the latest
// end); both slots start at all ones, and the launch took ~ts[1] - ts[0].
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
struct Stamp {
  unsigned long long *ts;
  __device__ __forceinline__ explicit Stamp(unsigned long long *p) : ts(p) {
    if (ts && threadIdx.x == 0) atomicMin(&ts[0], gtimer());
  }
  __device__ __forceinline__ ~Stamp() {
    if (ts && threadIdx.x == 0) atomicMin(&ts[1], ~gtimer());
  }
};

// BF16 storage trial: a value as a bfloat16 store would hold it (round to
// nearest even); binary64 plans never round.
__device__ __forceinline__ float rbf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ double rbf(double v) { return v; }
__device__ __forceinline__ float4 rbf4(const float4 &a) { return make_float4(rbf(a.x), rbf(a.y), rbf(a.z), rbf(a.w)); }

// Vector type of a 16-byte load, and its components by (unrolled) index.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };
__device__ __forceinline__ float vat(const float4 &v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
__device__ __forceinline__ double vat(const double2 &v, int c) { return c == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4 &v, int c, float a) {
  if (c == 0) v.x = a; else if (c == 1) v.y = a; else if (c == 2) v.z = a; else v.w = a;
}
__device__ __forceinline__ void vset(double2 &v, int c, double a) {
  if (c == 0) v.x = a; else v.y = a;
}

__device__ __forceinline__ float4 ld4(const float *p, int64_t i) { return *reinterpret_cast<const float4 *>(p + i); }
__device__ __forceinline__ void st4(float *p, int64_t i, const float4 &v) { *reinterpret_cast<float4 *>(p + i) = v; }

// --------------------------------------------------------------------------
// x-update right-hand side and warm residual
// --------------------------------------------------------------------------
// Partial sums of the grid-point launches: slot 0 holds r_0.r_0 of the
// right-hand side launch; the CG launch of phase ph (1 = w_0, 2, 3, ... = the
// steps) writes slot 1 + (ph & 1) and reads the slot of phase ph - 1.  A slot
// has nt_part entries per quantity (the right-hand side may use its own work
// items); a launch writes entry tl.seq of each of its work items and the
// entries past them stay zero.
template <typename A, typename D>
__device__ __forceinline__ A *cg_part(const D &in, int slot, int q) {
  return (A *)in.cgp + (int64_t)(slot * 2 + q) * in.nt_part;
}

// Rows of a segment that meet at grid point g in (A^T u)[g] (Eq. FD_mat):
// (A^T u)[g] = (u[ra] if va) - (u[rb] if vb), times 1/h for a difference.
struct AdjRows {
  int64_t ra, rb;
  bool va, vb;
};
__device__ __forceinline__ AdjRows adj_rows(const InstDev &in, int kind, const GridPos &p, int64_t g) {
  AdjRows a;
  switch (kind) {
    case SEG_DZ: {
      const int64_t r = g - p.t;  // iz + (nz-1)*t
      a.ra = r - 1;
      a.rb = r;
      a.va = p.iz >= 1;
      a.vb = p.iz <= in.nz - 2;
      break;
    }
    case SEG_DX: {
      const int64_t r = g - (int64_t)in.nz * p.iy;  // iz + nz*(ix + (nx-1)*iy)
      a.ra = r - in.nz;
      a.rb = r;
      a.va = p.ix >= 1;
      a.vb = p.ix <= in.nx - 2;
      break;
    }
    case SEG_DY: {
      a.ra = g - (int64_t)in.nz * in.nx;
      a.rb = g;
      a.va = p.iy >= 1;
      a.vb = p.iy <= in.ny - 2;
      break;
    }
    default:
      a.ra = g;
      a.rb = g;
      a.va = true;
      a.vb = false;
      break;
  }
  return a;
}

// b = sum_i A_i^T (rho_i y_i + v_i) (+ m in the direct form) and r = b - C x
// at the work item's grid points.  I is the index type of grid points and
// rows (32-bit while N < 2^31).
template <typename T, typename I, bool BL = false>
__device__ __forceinline__ void body_rhs_t(const Tile &tl, const InstDev &in, InstScal &sc) {
  using A = typename AccOf<T>::type;
  // points per thread per round, segments whose rows are loaded together
  // (the adds wait on the loads: batching the segments overlaps their
  // round trips)
  constexpr int PT = 2;
  constexpr int SB = sizeof(T) == 4 ? 4 : 2;
  constexpr int SUB = kThreads * PT;
  const int done = sc.done;
  const T *__restrict__ x = (const T *)in.x;
  const T *__restrict__ m = (const T *)in.m;
  T *__restrict__ r = (T *)in.cr[0];
  CSys<T> C;
  C.load(sc);
  // the segments with rows (the x-history ring, always the last segment,
  // has none): row arrays, kind, rho of the block, 1/h of the axis
  __shared__ const T *sy[kMaxSegs], *sv[kMaxSegs];
  __shared__ T srs[kMaxSegs], sih[kMaxSegs];
  __shared__ int skind[kMaxSegs];
  const int nseg = in.nseg - (in.nseg > 0 && in.seg[in.nseg - 1].kind == SEG_RING ? 1 : 0);
  if (threadIdx.x < nseg) {
    const SegDev &sg = in.seg[threadIdx.x];
    const int64_t bs = in.blk[sg.block].yoff + sg.row0;
    sy[threadIdx.x] = (const T *)in.y + bs;
    sv[threadIdx.x] = (const T *)in.v + bs;
    skind[threadIdx.x] = sg.kind;
    srs[threadIdx.x] = SV<T>::blk(sc, sg.block, BF_RHO);
    sih[threadIdx.x] = seg_ih<T>(in, sg.kind);
  }
  __syncthreads();
  if (done) return;
  const int alg1 = in.alg1;
  const I nz = (I)in.nz, sxy = (I)in.nz * (I)in.nx;
  const I end = (I)(tl.start + tl.len);
  A a1 = A(0);
  for (I base = (I)tl.start; base < end; base += SUB) {
    I g[PT], rz[PT], rx[PT];
    bool fza[PT], fzb[PT], fxa[PT], fxb[PT], fya[PT], fyb[PT];
    T b[PT];
    Nbr<T> xn[PT];
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      g[e] = base + (I)threadIdx.x + (I)(e * kThreads);
      b[e] = T(0);
      if (g[e] < end) {
        const GridPos pos = grid_pos(in, g[e]);
        if (!alg1) b[e] = m[g[e]];
        load_nbr<T>(in, pos, g[e], [&](int64_t i) { return x[i]; }, xn[e]);
        // rows of the difference operators meeting at g (Eq. FD_mat)
        rz[e] = g[e] - (I)pos.t;         // D_z: iz + (nz-1) t
        rx[e] = g[e] - nz * (I)pos.iy;   // D_x: iz + nz (ix + (nx-1) iy)
        fza[e] = pos.iz >= 1;
        fzb[e] = pos.iz <= in.nz - 2;
        fxa[e] = pos.ix >= 1;
        fxb[e] = pos.ix <= in.nx - 2;
        fya[e] = pos.iy >= 1;
        fyb[e] = pos.iy <= in.ny - 2;
      } else {
        rz[e] = rx[e] = 0;
        fza[e] = fzb[e] = fxa[e] = fxb[e] = fya[e] = fyb[e] = false;
      }
    }
    for (int s0 = 0; s0 < nseg; s0 += SB) {
      T ya[SB][PT], va[SB][PT], yb[SB][PT], vb[SB][PT];
#pragma unroll
      for (int j = 0; j < SB; ++j) {
        const int sgi = s0 + j;
        const bool live = sgi < nseg;
        const int kind = live ? skind[sgi] : SEG_RING;
        const T *__restrict__ ys = live ? sy[sgi] : nullptr;
        const T *__restrict__ vs = live ? sv[sgi] : nullptr;
#pragma unroll
        for (int e = 0; e < PT; ++e) {
          // (A^T u)[g] = u[ia] (if fa) - u[ib] (if fb), times 1/h
          I ia = g[e], ib = g[e];
          bool fa = false, fb = false;
          switch (kind) {
            case SEG_I: fa = g[e] < end; break;
            case SEG_DZ: ia = rz[e] - 1; ib = rz[e]; fa = fza[e]; fb = fzb[e]; break;
            case SEG_DX: ia = rx[e] - nz; ib = rx[e]; fa = fxa[e]; fb = fxb[e]; break;
            case SEG_DY: ia = g[e] - sxy; fa = fya[e]; fb = fyb[e]; break;
            default: break;
          }
          ya[j][e] = fa ? ys[ia] : T(0);
          va[j][e] = fa ? vs[ia] : T(0);
          yb[j][e] = fb ? ys[ib] : T(0);
          vb[j][e] = fb ? vs[ib] : T(0);
        }
      }
#pragma unroll
      for (int j = 0; j < SB; ++j) {
        const int sgi = s0 + j;
        if (sgi < nseg) {
          const T rho = srs[sgi], ih = sih[sgi];
#pragma unroll
          for (int e = 0; e < PT; ++e)
            b[e] += ((rho * ya[j][e] + va[j][e]) - (rho * yb[j][e] + vb[j][e])) * ih;
        }
      }
    }
    if constexpr (BL) {
      // the blur block's F^T (rho y + v) - rho F^T F x (blur right-hand side launch)
      if (in.bl_R) {
        const T *__restrict__ t = (const T *)in.bl_s;
#pragma unroll
        for (int e = 0; e < PT; ++e)
          if (g[e] < end) b[e] += t[g[e]];
      }
    }
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      if (g[e] < end) {
        const T rv = b[e] - apply_c(C, xn[e]);
        r[g[e]] = rv;
        a1 += (A)rv * (A)rv;
      }
    }
  }
  A acc[1] = {a1};
  block_sum<1>(acc);
  if (threadIdx.x == 0) cg_part<A>(in, 0, 0)[tl.seq] = acc[0];
}

template <typename T, bool BL = false>
__device__ __forceinline__ void body_rhs(const Tile &tl, const InstDev *__restrict__ insts,
                                         InstScal *__restrict__ scal) {
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= in.N, 1u, tl.start + tl.len);
  if (in.N <= (int64_t)0x7fffffff)
    body_rhs_t<T, int, BL>(tl, in, sc);
  else
    body_rhs_t<T, int64_t, BL>(tl, in, sc);
}

// w_0 of the blur block items (defined with the CG launches below)
template <typename T>
__device__ void body_cg_w0_blur(const Tile &tl, const InstDev &in, InstScal &sc);

template <typename T, bool ONE, bool BL = false>
__global__ void __launch_bounds__(kThreads, 3) k_rhs(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                  InstScal *__restrict__ scal, unsigned long long *ts,
                                                  const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  body_rhs<T, BL>(tiles[blockIdx.x], ONE ? &one.d : insts, scal);
}

// --------------------------------------------------------------------------
// Staged right-hand side (binary32, 2D): the y and v rows every segment's
// adjoint reads at this work item's grid points are contiguous windows;
// one thread moves them into shared memory with bulk copies (the TMA
// engine, completion counted in bytes on an mbarrier) while the CTA loads
// its x stencil, then the adjoint differences read shared memory only.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy; both addresses and the size multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// true once phase `parity` of the barrier completed, false after `polls` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long polls) {
  for (long long i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
constexpr long long kBulkWaitPolls = 1ll << 22;

// Rows of the window a segment's adjoint reads at grid points [s, e) of a
// 2D grid (Eq. FD_mat), segment-relative, [lo, hi) inside [0, M).
__device__ __forceinline__ void rhs_window(const InstDev &in, int kind, int64_t M, int64_t s, int64_t e, int64_t &lo,
                                           int64_t &hi) {
  switch (kind) {
    case SEG_DZ: {  // rows g - g / n_z; a = r - 1, b = r
      lo = s - (int64_t)fdiv((uint32_t)s, in.fz) - 1;
      hi = (e - 1) - (int64_t)fdiv((uint32_t)(e - 1), in.fz) + 1;
      break;
    }
    case SEG_DX:  // rows g (2D); a = g - n_z, b = g
      lo = s - in.nz;
      hi = e;
      break;
    default:  // identity: rows g
      lo = s;
      hi = e;
      break;
  }
  if (lo < 0) lo = 0;
  if (hi > M) hi = M;
  if (hi < lo) hi = lo;
}

template <bool ONE>
__global__ void __launch_bounds__(kThreads, 2) k_rhs_tma(const Tile *__restrict__ tiles,
                                                         const InstDev *__restrict__ insts_g,
                                                         InstScal *__restrict__ scal, unsigned long long *ts,
                                                         const __grid_constant__ InstOne one) {
  const InstDev *__restrict__ insts = ONE ? &one.d : insts_g;
  const Stamp stamp(ts);
  extern __shared__ __align__(128) float sw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int sbase_y[kMaxSegs], sbase_v[kMaxSegs];  // shared index of row 0 of each segment
  __shared__ int64_t sg0[kMaxSegs], sgn[kMaxSegs];      // window: first absolute row, rows (multiples of 4)
  __shared__ float srs[kMaxSegs], sih[kMaxSegs];
  __shared__ int skind[kMaxSegs];
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= in.N, 1u, tl.start + tl.len);
  const int done = sc.done;
  const float *__restrict__ x = (const float *)in.x;
  const float *__restrict__ m = (const float *)in.m;
  const float *__restrict__ y = (const float *)in.y;
  const float *__restrict__ v = (const float *)in.v;
  float *__restrict__ r = (float *)in.cr[0];
  const int nseg = in.nseg - (in.nseg > 0 && in.seg[in.nseg - 1].kind == SEG_RING ? 1 : 0);
  const int64_t s0 = tl.start, e0 = tl.start + tl.len;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  if (threadIdx.x < nseg) {
    const SegDev &sg = in.seg[threadIdx.x];
    const int64_t bs = in.blk[sg.block].yoff + sg.row0;
    int64_t lo, hi;
    rhs_window(in, sg.kind, sg.len, s0, e0, lo, hi);
    const int64_t a0 = (bs + lo) & ~(int64_t)3, a1 = (bs + hi + 3) & ~(int64_t)3;
    sg0[threadIdx.x] = a0;
    sgn[threadIdx.x] = hi > lo ? a1 - a0 : 0;
    skind[threadIdx.x] = sg.kind;
    srs[threadIdx.x] = SV<float>::blk(sc, sg.block, BF_RHO);
    sih[threadIdx.x] = seg_ih<float>(in, sg.kind);
    // row i of the segment sits at shared index (window offset) + bs - a0 + i;
    // bs - a0 is about -lo, so the base may lie before the window
    sbase_y[threadIdx.x] = (int)(bs - a0);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  if (done) return;  // no copy was issued
  if (threadIdx.x == 0) {
    // y windows back to back, then the v windows
    int64_t tot = 0;
    for (int j = 0; j < nseg; ++j) tot += sgn[j];
    mbar_expect_tx(&bar, (uint32_t)(2 * tot * sizeof(float)));
    int64_t oy = 0;
    for (int j = 0; j < nseg; ++j) {
      const int64_t n = sgn[j];
      if (n) {
        bulk_g2s(sw + oy, y + sg0[j], (uint32_t)(n * sizeof(float)), &bar);
        bulk_g2s(sw + tot + oy, v + sg0[j], (uint32_t)(n * sizeof(float)), &bar);
      }
      sbase_v[j] = (int)(tot + oy) + sbase_y[j];
      sbase_y[j] += (int)oy;
      oy += n;
    }
  }
  CSys<float> C;
  C.load(sc);
  const int alg1 = in.alg1;
  const int nz = in.nz;
  float a1 = 0.f;
  bool waited = false;
  // U grid points per thread per round (g, g + kThreads, ...): their x
  // stencils and m are requested together. Every thread runs the same
  // rounds (at least one), and the first round waits for the copies.
  constexpr int U = 4;
  for (int64_t base = s0; base < e0 || !waited; base += (int64_t)kThreads * U) {
    GridPos pos[U];
    Nbr<float> xn[U];
    float b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t g = base + threadIdx.x + (int64_t)u * kThreads;
      b[u] = 0.f;
      if (g < e0) {
        pos[u] = grid_pos(in, g);
        if (!alg1) b[u] = m[g];
        load_nbr<float>(in, pos[u], g, [&](int64_t i) { return x[i]; }, xn[u]);
      }
    }
    if (!waited) {
      __syncthreads();  // sbase_* written by thread 0
      const bool late = !mbar_wait(&bar, 0, kBulkWaitPolls);
      if (__syncthreads_or(late)) {  // the same decision in every thread
        if (threadIdx.x == 0) atomicExch(in.err, (uint32_t)SIP_ERR_TIMEOUT);
        mbar_wait(&bar, 0, kBulkWaitPolls);  // the copies in flight land before the CTA ends
        return;
      }
      waited = true;
    }
    // segments outside, this thread's points inside: a segment's descriptor
    // is read once per round and its kind decides the loop taken (each
    // point still adds its segments in order)
    int gi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) gi[u] = (int)(base + threadIdx.x + (int64_t)u * kThreads);
    for (int j = 0; j < nseg; ++j) {
      const float *__restrict__ ys = sw + sbase_y[j];
      const float *__restrict__ vs = sw + sbase_v[j];
      const float rho = srs[j], ih = sih[j];
      const int kind = skind[j];
      // (A^T u)[g] = u[ia] (if fa) - u[ib] (if fb), times 1/h
      if (kind == SEG_DZ) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (gi[u] >= e0) continue;
          const int rz = gi[u] - (int)pos[u].t;  // D_z row base (iz + (nz-1) t)
          const float ua = pos[u].iz >= 1 ? rho * ys[rz - 1] + vs[rz - 1] : 0.f;
          const float ub = pos[u].iz <= nz - 2 ? rho * ys[rz] + vs[rz] : 0.f;
          b[u] += (ua - ub) * ih;
        }
      } else if (kind == SEG_DX) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (gi[u] >= e0) continue;
          const int ia = gi[u] - nz;
          const float ua = pos[u].ix >= 1 ? rho * ys[ia] + vs[ia] : 0.f;
          const float ub = pos[u].ix <= in.nx - 2 ? rho * ys[gi[u]] + vs[gi[u]] : 0.f;
          b[u] += (ua - ub) * ih;
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (gi[u] >= e0) continue;
          const float ua = rho * ys[gi[u]] + vs[gi[u]], ub = 0.f;
          b[u] += (ua - ub) * ih;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (gi[u] >= e0) continue;
      const float rv = b[u] - apply_c(C, xn[u]);
      r[gi[u]] = rv;
      a1 += rv * rv;
    }
  }
  float acc[1] = {a1};
  block_sum<1>(acc);
  if (threadIdx.x == 0) cg_part<float>(in, 0, 0)[tl.seq] = acc[0];
}

// --------------------------------------------------------------------------
// Conjugate gradient on C x = b from the warm start x (Sec. "Solving the
// linear system and automatic parameter selection"), in the Chronopoulos-Gear
// arrangement of the CG recurrences: with w = C r and s = C p kept as
// vectors, both inner products of a step (gamma = r.r, delta = w.r) come
// from one reduction, so a step is one launch:
//   p_i = r_i + beta_i p_{i-1};      s_i = w_i + beta_i s_{i-1}
//   x_{i+1} = x_i + alpha_i p_i;     r_{i+1} = r_i - alpha_i s_i
//   w_{i+1} = C r_{i+1};  gamma_{i+1} = r_{i+1}.r_{i+1};  delta_{i+1} = w_{i+1}.r_{i+1}
//   beta_{i+1} = gamma_{i+1} / gamma_i
//   alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i)
// In exact arithmetic these are the iterates of textbook CG; the
// denominator of alpha equals p^T C p, so "p^T C p <= 0" stops as in CG.
// No launch finalises its own sums: each CTA of the next launch adds the
// per-tile partials (the same bits in every CTA) and derives alpha, beta.
// The r, w, s buffers alternate with the launch: the right-hand side and
// w_0 use buffer 0, the step launch of phase ph reads buffer ph & 1 and
// writes the other one.
// --------------------------------------------------------------------------
// w_0 = C r_0 on 2D grids with n_z % 4 == 0 and aligned arrays: 4
// consecutive z samples per thread, z neighbours across lanes (single
// loads at warp and tile edges), as in the four-sample CG step.
template <typename D>
__device__ __forceinline__ void body_cg_w0_v4(const Tile &tl, const D &in, const InstScal &sc, int done) {
  constexpr int SUB = kThreads * 4;
  const unsigned FULL = 0xffffffffu;
  const float *__restrict__ r = (const float *)in.cr[0];
  float *__restrict__ w = (float *)in.cw[0];
  CSys<float> C;
  C.load(sc);
  const int lane = threadIdx.x & 31;
  const int64_t end = tl.start + tl.len;
  float a0 = 0.f;
  for (int64_t base = tl.start; base < end; base += SUB) {
    const int64_t g0 = base + 4 * (int64_t)threadIdx.x;
    const bool ok = g0 < end;
    float4 R = make_float4(0.f, 0.f, 0.f, 0.f), RXM = R, RXP = R;
    float zm = 0.f, zp = 0.f;
    bool hzm = false, hzp = false, edge_p = false;
    if (ok) {
      const GridPos ps = grid_pos(in, g0);
      R = ld4(r, g0);
      RXM = ps.ix > 0 ? ld4(r, g0 - in.nz) : R;
      RXP = ps.ix < in.nx - 1 ? ld4(r, g0 + in.nz) : R;
      hzm = ps.iz > 0;
      hzp = ps.iz + 4 < in.nz;
      edge_p = lane == 31 || g0 + 4 >= end;
      if (hzm && lane == 0) zm = r[g0 - 1];
      if (hzp && edge_p) zp = r[g0 + 4];
    }
    const float um = __shfl_up_sync(FULL, R.w, 1), up = __shfl_down_sync(FULL, R.x, 1);
    if (done) return;
    if (!ok) continue;
    if (lane != 0) zm = um;
    if (!edge_p) zp = up;
    if (!hzm) zm = R.x;
    if (!hzp) zp = R.w;
    Nbr<float> nb;
    float4 W;
    nb = {R.x, zm, R.y, RXM.x, RXP.x, R.x, R.x};
    W.x = apply_c(C, nb);
    nb = {R.y, R.x, R.z, RXM.y, RXP.y, R.y, R.y};
    W.y = apply_c(C, nb);
    nb = {R.z, R.y, R.w, RXM.z, RXP.z, R.z, R.z};
    W.z = apply_c(C, nb);
    nb = {R.w, R.z, zp, RXM.w, RXP.w, R.w, R.w};
    W.w = apply_c(C, nb);
    st4(w, g0, W);
    a0 += W.x * R.x + W.y * R.y + W.z * R.z + W.w * R.w;
  }
  float acc[1] = {a0};
  block_sum<1>(acc);
  if (threadIdx.x == 0) cg_part<float>(in, 2, 0)[tl.seq] = acc[0];  // delta_0 = r_0^T C r_0
}

template <typename T, typename D>
__device__ __forceinline__ void body_cg_w0_in(const Tile &tl, const D &in, InstScal &sc) {
  SIP_STEP_CONSTANTS;
  using A = typename AccOf<T>::type;
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= in.N, 2u, tl.start + tl.len);
  const int done = sc.done;
  if constexpr (sizeof(T) == 4) {
    if ((in.nz & 3) == 0 && in.ny == 1 && (((uintptr_t)in.cr[0] | (uintptr_t)in.cw[0]) & 15) == 0) {
      body_cg_w0_v4(tl, in, sc, done);
      return;
    }
  }
  const T *__restrict__ r = (const T *)in.cr[0];
  T *__restrict__ w = (T *)in.cw[0];
  CSys<T> C;
  C.load(sc);
  const int64_t end = tl.start + tl.len;
  A a0 = A(0);
  for (int64_t base = tl.start; base < end; base += SUB) {
    Nbr<T> rn[PT];
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) load_nbr<T>(in, grid_pos(in, g), g, [&](int64_t i) { return r[i]; }, rn[e]);
    }
    if (done) return;
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) {
        const T wg = apply_c(C, rn[e]);
        w[g] = wg;
        a0 += (A)wg * (A)rn[e].c;
      }
    }
  }
  A acc[1] = {a0};
  block_sum<1>(acc);
  if (threadIdx.x == 0) cg_part<A>(in, 2, 0)[tl.seq] = acc[0];  // delta_0 = r_0^T C r_0 = p_0^T C p_0
}
template <typename T>
__device__ __forceinline__ void body_cg_w0(const Tile &tl, const InstDev *__restrict__ insts,
                                           InstScal *__restrict__ scal) {
  body_cg_w0_in<T>(tl, insts[tl.inst], scal[tl.inst]);
}

// Single-instance plans: the grid-point work item of CTA b (items of `chunk`
// points from 0) and the CG's descriptor fields arrive as launch parameters,
// so a CG launch starts loading without first reading its item and the
// instance descriptor from memory.
__device__ __forceinline__ Tile one_tile(const CgOne &one) {
  Tile tl;
  tl.inst = 0;
  tl.item = 0;
  tl.start = (int64_t)blockIdx.x * one.chunk;
  const int64_t left = one.d.N - tl.start;
  tl.len = (int32_t)(left < one.chunk ? left : one.chunk);
  tl.seq = (int32_t)blockIdx.x;
  return tl;
}

template <typename T, bool BL = false>
__global__ void __launch_bounds__(kThreads, 4) k_cg_w0(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                       InstScal *__restrict__ scal, unsigned long long *ts,
                                                       const __grid_constant__ CgOne one) {
  const Stamp stamp(ts);
  if constexpr (BL) {
    if (!one.on && tiles[blockIdx.x].item > 0) {
      const Tile tl = tiles[blockIdx.x];
      body_cg_w0_blur<T>(tl, insts[tl.inst], scal[tl.inst]);
      return;
    }
  }
  if (one.on)
    body_cg_w0_in<T>(one_tile(one), one.d, scal[0]);
  else
    body_cg_w0<T>(tiles[blockIdx.x], insts, scal);
}

// CG state fields in the storage precision (binary32 kernels do their
// scalar work in binary32: binary64 issues at a small fraction of the rate).
template <typename T> struct CgOf;
template <> struct CgOf<double> {
  static __device__ __forceinline__ double &alpha(CgState &s) { return s.alpha; }
  static __device__ __forceinline__ double &rr(CgState &s) { return s.rr; }
  static __device__ __forceinline__ double &rr0(CgState &s) { return s.rr0; }
};
template <> struct CgOf<float> {
  static __device__ __forceinline__ float &alpha(CgState &s) { return s.alphaf; }
  static __device__ __forceinline__ float &rr(CgState &s) { return s.rrf; }
  static __device__ __forceinline__ float &rr0(CgState &s) { return s.rr0f; }
};

// alpha, beta and "take a step" for the step launch of phase ph >= 2: all
// threads add the partial sums, thread 0 updates the CG state (the same
// values in every CTA) and the instance's first tile stores it for the next
// launch.  Results in s_ab, s_go after the closing __syncthreads.
// The partial sums a step launch of phase ph gathers (binary32 storage):
// pointers of the two quantities.
template <typename D>
__device__ __forceinline__ void cg_gather_src(const D &in, int ph, const float *(&p)[2]) {
  const int slot = 1 + ((ph - 1) & 1);
  p[0] = ph == 2 ? cg_part<float>(in, 0, 0) : cg_part<float>(in, slot, 0);
  p[1] = ph == 2 ? cg_part<float>(in, 2, 0) : cg_part<float>(in, slot, 1);
}

// pre (binary32): the first batch of the partial sums, requested by
// gather_first before the launch's data loads (or null)
template <typename T, typename D>
__device__ __forceinline__ void cg_scalars(const Tile &tl, const D &in, InstScal &sc, int ph, T *s_ab,
                                           int *s_go, const float (*pre)[kGatherBatch] = nullptr) {
  using A = typename AccOf<T>::type;
  using G = CgOf<T>;
  const int nt = in.nt_part;  // entries past a launch's own work items stay zero
  const int done = *(volatile const int *)&sc.done;
  T t[2] = {T(0), T(0)};
  CgState *pv = &sc.cg[(ph - 1) & 1];
  int prev_active = 1;
  if (ph == 2) {
    // r_0.r_0 from the right-hand side launch, delta_0 from the w_0 launch
    const A *const p[2] = {cg_part<A>(in, 0, 0), cg_part<A>(in, 2, 0)};
    if (!done) {
      if constexpr (sizeof(T) == 4)
        cta_gather<2>(p, nt, t, pre);
      else
        cta_gather<2>(p, nt, t);
    }
  } else {
    prev_active = __ldcg(&pv->active);
    const int slot = 1 + ((ph - 1) & 1);
    const A *const p[2] = {cg_part<A>(in, slot, 0), cg_part<A>(in, slot, 1)};
    if (!done && prev_active) {
      if constexpr (sizeof(T) == 4)
        cta_gather<2>(p, nt, t, pre);
      else
        cta_gather<2>(p, nt, t);
    }
  }
  if (threadIdx.x == 0) {
    CgState st;
    T beta = T(0);
    if (ph == 2) {
      const T rr0 = t[0], delta = t[1];
      const int limit = in.cg_iters > 0 ? in.cg_iters : in.cg_max;
      st.active = (limit > 0 && rr0 > T(0) && delta > T(0)) ? 1 : 0;
      G::alpha(st) = st.active ? rr0 / delta : T(0);
      G::rr(st) = rr0;
      G::rr0(st) = rr0;
      st.steps = 0;
    } else {
      G::alpha(st) = __ldcg(&G::alpha(*pv));
      G::rr(st) = __ldcg(&G::rr(*pv));
      G::rr0(st) = __ldcg(&G::rr0(*pv));
      st.steps = __ldcg(&pv->steps);
      st.active = prev_active;
      if (st.active) {
        const T g1 = t[0], d1 = t[1];
        st.steps += 1;
        bool more;
        if (in.cg_iters > 0) {
          more = st.steps < in.cg_iters;
        } else {  // Eq. cg_stop: ||r_j|| < 0.1 ||r_0||
          more = st.steps < in.cg_max && !(sqrt(g1) < T(0.1) * sqrt(G::rr0(st)));
        }
        const T b1 = g1 / G::rr(st);
        const T den = d1 - b1 * g1 / G::alpha(st);  // = p_{i+1}^T C p_{i+1}
        if (more && g1 > T(0) && den > T(0)) {
          beta = b1;
          G::alpha(st) = g1 / den;
        } else {
          st.active = 0;
        }
        G::rr(st) = g1;
      }
    }
    s_ab[0] = G::alpha(st);
    s_ab[1] = beta;
    *s_go = (st.active && !done) ? 1 : 0;
    if (tl.seq == 0 && !done) {
      pv = &sc.cg[ph & 1];
      G::alpha(*pv) = G::alpha(st);
      G::rr(*pv) = G::rr(st);
      G::rr0(*pv) = G::rr0(st);
      pv->active = st.active;
      pv->steps = st.steps;
    }
  }
  __syncthreads();
}

// Binary32 CG step on 2D grids with n_z % 4 == 0 (so every column starts on
// a multiple of 4) whose arrays start on 16-byte boundaries: a thread takes
// 4 consecutive z samples of one column with 16-byte loads and stores; the
// z neighbours beyond its 4 come from the adjacent lanes, or, at a warp or
// tile edge, from single loads.  Same arithmetic per sample as the general
// step.  FIRST (the first step, beta = 0): p and s_{i-1} are taken as zero
// instead of being read (beta times them is zero).
template <bool FIRST, typename D>
__device__ __forceinline__ void body_cg_step_v4(const Tile &tl, const D &in, InstScal &sc, int ph) {
  constexpr int SUB = kThreads * 4;
  const unsigned FULL = 0xffffffffu;
  const int c = ph & 1, n = c ^ 1;
  const float *__restrict__ r = (const float *)in.cr[c];
  const float *__restrict__ w = (const float *)in.cw[c];
  const float *__restrict__ sp = (const float *)in.cs[c];  // s_{i-1}
  float *__restrict__ rn_ = (float *)in.cr[n];
  float *__restrict__ wn_ = (float *)in.cw[n];
  float *__restrict__ sn_ = (float *)in.cs[n];             // s_i
  float *__restrict__ p = (float *)in.cp;
  float *__restrict__ x = (float *)in.x;
  __shared__ float s_ab[2];
  __shared__ int s_go;
  float alpha = 0.f, beta = 0.f;
  CSys<float> C;
  C.load(sc);
  const int lane = threadIdx.x & 31;
  const int64_t end = tl.start + tl.len;  // a multiple of 4
  float ag = 0.f, ad = 0.f;
  for (int64_t base = tl.start; base < end; base += SUB) {
    const int64_t g0 = base + 4 * (int64_t)threadIdx.x;
    const bool ok = g0 < end;
    float4 rc, wc, sc4, pv, xv, rxm, wxm, sxm, rxp, wxp, sxp;
    float rzm = 0.f, wzm = 0.f, szm = 0.f, rzp = 0.f, wzp = 0.f, szp = 0.f;
    bool hzm = false, hzp = false, edge_p = false;
    if (ok) {
      const GridPos ps = grid_pos(in, g0);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      rc = ld4(r, g0);
      wc = ld4(w, g0);
      sc4 = FIRST ? z4 : ld4(sp, g0);
      pv = FIRST ? z4 : ld4(p, g0);
      xv = ld4(x, g0);
      // a missing neighbour repeats the centre, so its difference is zero
      const bool hxm = ps.ix > 0, hxp = ps.ix < in.nx - 1;
      rxm = hxm ? ld4(r, g0 - in.nz) : rc;
      wxm = hxm ? ld4(w, g0 - in.nz) : wc;
      sxm = (hxm && !FIRST) ? ld4(sp, g0 - in.nz) : sc4;
      rxp = hxp ? ld4(r, g0 + in.nz) : rc;
      wxp = hxp ? ld4(w, g0 + in.nz) : wc;
      sxp = (hxp && !FIRST) ? ld4(sp, g0 + in.nz) : sc4;
      hzm = ps.iz > 0;
      hzp = ps.iz + 4 < in.nz;
      edge_p = lane == 31 || g0 + 4 >= end;
      if (hzm && lane == 0) {
        rzm = r[g0 - 1];
        wzm = w[g0 - 1];
        szm = FIRST ? 0.f : sp[g0 - 1];
      }
      if (hzp && edge_p) {
        rzp = r[g0 + 4];
        wzp = w[g0 + 4];
        szp = FIRST ? 0.f : sp[g0 + 4];
      }
    }
    if (base == tl.start) {
      // the previous launch's sums, while this CTA's first loads are in flight
      cg_scalars<float>(tl, in, sc, ph, s_ab, &s_go);
      if (!s_go) return;
      alpha = s_ab[0];
      beta = s_ab[1];
    }
    // r_{i+1} = r_i - alpha (w_i + beta s_{i-1}) at the samples and their neighbours
    auto nr = [&](float rv, float wv, float sv) { return rv - alpha * (wv + beta * sv); };
    auto nr4 = [&](const float4 &a, const float4 &b, const float4 &d) {
      return make_float4(nr(a.x, b.x, d.x), nr(a.y, b.y, d.y), nr(a.z, b.z, d.z), nr(a.w, b.w, d.w));
    };
    float4 R = ok ? nr4(rc, wc, sc4) : make_float4(0.f, 0.f, 0.f, 0.f);
    float zm = __shfl_up_sync(FULL, R.w, 1), zp = __shfl_down_sync(FULL, R.x, 1);
    if (!ok) continue;
    const float4 RXM = nr4(rxm, wxm, sxm), RXP = nr4(rxp, wxp, sxp);
    if (lane == 0) zm = nr(rzm, wzm, szm);
    if (edge_p) zp = nr(rzp, wzp, szp);
    if (!hzm) zm = R.x;
    if (!hzp) zp = R.w;
    Nbr<float> nb;
    float4 W;
    nb = {R.x, zm, R.y, RXM.x, RXP.x, R.x, R.x};
    W.x = apply_c(C, nb);
    nb = {R.y, R.x, R.z, RXM.y, RXP.y, R.y, R.y};
    W.y = apply_c(C, nb);
    nb = {R.z, R.y, R.w, RXM.z, RXP.z, R.z, R.z};
    W.z = apply_c(C, nb);
    nb = {R.w, R.z, zp, RXM.w, RXP.w, R.w, R.w};
    W.w = apply_c(C, nb);
    const float4 S = make_float4(wc.x + beta * sc4.x, wc.y + beta * sc4.y, wc.z + beta * sc4.z, wc.w + beta * sc4.w);
    const float4 Pn = make_float4(rc.x + beta * pv.x, rc.y + beta * pv.y, rc.z + beta * pv.z, rc.w + beta * pv.w);
    st4(p, g0, Pn);
    st4(x, g0, make_float4(xv.x + alpha * Pn.x, xv.y + alpha * Pn.y, xv.z + alpha * Pn.z, xv.w + alpha * Pn.w));
    st4(sn_, g0, S);
    st4(rn_, g0, R);
    st4(wn_, g0, W);
    ag += R.x * R.x + R.y * R.y + R.z * R.z + R.w * R.w;
    ad += W.x * R.x + W.y * R.y + W.z * R.z + W.w * R.w;
  }
  float acc[2] = {ag, ad};
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    const int slot = 1 + (ph & 1);
    cg_part<float>(in, slot, 0)[tl.seq] = acc[0];
    cg_part<float>(in, slot, 1)[tl.seq] = acc[1];
  }
}

template <typename T, typename D, bool FIRST = false>
__device__ __forceinline__ void body_cg_step_in(const Tile &tl, const D &in, InstScal &sc, int ph) {
  using A = typename AccOf<T>::type;
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= in.N, 3u, tl.start + tl.len);
  constexpr int PT = sizeof(T) == 4 ? 2 : 1;  // 3 stencils per row: keep the register budget
  constexpr int SUB = kThreads * PT;
  if constexpr (sizeof(T) == 4) {
    // 16-byte accesses need every array on a 16-byte boundary (the x of a
    // batched plan is packed and may not be)
    const uintptr_t al = (uintptr_t)in.x | (uintptr_t)in.cp | (uintptr_t)in.cr[0] | (uintptr_t)in.cr[1] |
                         (uintptr_t)in.cw[0] | (uintptr_t)in.cw[1] | (uintptr_t)in.cs[0] | (uintptr_t)in.cs[1];
    if ((in.nz & 3) == 0 && in.ny == 1 && (al & 15) == 0) {
      body_cg_step_v4<FIRST>(tl, in, sc, ph);  // FIRST (beta = 0): p and s_{i-1} are not read
      return;
    }
  }
  const int c = ph & 1, n = c ^ 1;
  const T *__restrict__ r = (const T *)in.cr[c];
  const T *__restrict__ w = (const T *)in.cw[c];
  const T *__restrict__ sp = (const T *)in.cs[c];  // s_{i-1}
  T *__restrict__ rn_ = (T *)in.cr[n];
  T *__restrict__ wn_ = (T *)in.cw[n];
  T *__restrict__ sn_ = (T *)in.cs[n];             // s_i
  T *__restrict__ p = (T *)in.cp;
  T *__restrict__ x = (T *)in.x;
  __shared__ T s_ab[2];
  __shared__ int s_go;
  T alpha = T(0), beta = T(0);
  CSys<T> C;
  C.load(sc);
  const int64_t end = tl.start + tl.len;
  A ag = A(0), ad = A(0);
  for (int64_t base = tl.start; base < end; base += SUB) {
    Nbr<T> rr[PT], ww[PT], ss[PT];
    T pv[PT], xv[PT];
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) {
        const GridPos ps = grid_pos(in, g);
        load_nbr<T>(in, ps, g, [&](int64_t i) { return r[i]; }, rr[e]);
        load_nbr<T>(in, ps, g, [&](int64_t i) { return w[i]; }, ww[e]);
        load_nbr<T>(in, ps, g, [&](int64_t i) { return sp[i]; }, ss[e]);
        pv[e] = p[g];
        xv[e] = x[g];
      }
    }
    if (base == tl.start) {
      // the previous launch's sums, while this CTA's first loads are in flight
      cg_scalars<T>(tl, in, sc, ph, s_ab, &s_go);
      if (!s_go) return;
      alpha = s_ab[0];
      beta = s_ab[1];
    }
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) {
        // s_i and r_{i+1} at the stencil points (a missing neighbour repeats
        // the centre, so its difference stays zero)
        Nbr<T> rnew;
        const T s_c = ww[e].c + beta * ss[e].c;
        rnew.c = rr[e].c - alpha * s_c;
#define SIP_CG_AT(f) rnew.f = rr[e].f - alpha * (ww[e].f + beta * ss[e].f);
        SIP_CG_AT(zm)
        SIP_CG_AT(zp)
        SIP_CG_AT(xm)
        SIP_CG_AT(xp)
        SIP_CG_AT(ym)
        SIP_CG_AT(yp)
#undef SIP_CG_AT
        const T pi = rr[e].c + beta * pv[e];
        p[g] = pi;
        x[g] = xv[e] + alpha * pi;
        sn_[g] = s_c;
        rn_[g] = rnew.c;
        const T wnew = apply_c(C, rnew);
        wn_[g] = wnew;
        ag += (A)rnew.c * (A)rnew.c;
        ad += (A)wnew * (A)rnew.c;
      }
    }
  }
  A acc[2] = {ag, ad};
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    const int slot = 1 + (ph & 1);
    cg_part<A>(in, slot, 0)[tl.seq] = acc[0];
    cg_part<A>(in, slot, 1)[tl.seq] = acc[1];
  }
}

template <typename T>
__device__ __forceinline__ void body_cg_step(const Tile &tl, const InstDev *__restrict__ insts,
                                             InstScal *__restrict__ scal, int ph) {
  body_cg_step_in<T>(tl, insts[tl.inst], scal[tl.inst], ph);
}

// out of line: the single-instance path keeps the register allocation
template <typename T>
__device__ __noinline__ void cg_step_call(const Tile &tl, const InstDev *insts, InstScal *scal, int ph) {
  body_cg_step<T>(tl, insts, scal, ph);
}

// The last step launch of an iteration.  The next iteration restarts the CG
// from r_0 = b - C x, so of this launch's results only
// x_{i+1} = x_i + alpha_i p_i, p_i = r_i + beta_i p_{i-1}, is read again: r, w,
// s, p and the partial sums are not formed (4 words per grid point instead
// of 10, no stencil).  alpha_i, beta_i and the CG state come from the same
// gather as in a full step, so the iterate is the full step's.
template <typename T, typename D>
__device__ __forceinline__ void body_cg_last_in(const Tile &tl, const D &in, InstScal &sc, int ph) {
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= in.N, 3u, tl.start + tl.len);
  const int c = ph & 1;
  const T *__restrict__ r = (const T *)in.cr[c];
  const T *__restrict__ p = (const T *)in.cp;
  T *__restrict__ x = (T *)in.x;
  __shared__ T s_ab[2];
  __shared__ int s_go;
  const int64_t end = tl.start + tl.len;
  T alpha = T(0), beta = T(0);
  bool first = true;
  if constexpr (sizeof(T) == 4) {
    const uintptr_t al = (uintptr_t)(r + tl.start) | (uintptr_t)(p + tl.start) | (uintptr_t)(x + tl.start);
    if ((al & 15) == 0 && (tl.len & 3) == 0) {
      // the partial sums are requested before the data, so that their sum
      // is formed while the data loads are in flight
      const float *gp[2];
      cg_gather_src(in, ph, gp);
      float pre[2][kGatherBatch];
      gather_first<2>(gp, in.nt_part, pre);
      for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * 4) {
        const int64_t g0 = base + 4 * (int64_t)threadIdx.x;
        const bool ok = g0 < end;
        float4 rv, pv, xv;
        if (ok) {
          rv = ld4(r, g0);
          pv = ld4(p, g0);
          xv = ld4(x, g0);
        }
        if (first) {
          cg_scalars<T>(tl, in, sc, ph, s_ab, &s_go, pre);
          if (!s_go) return;
          alpha = s_ab[0];
          beta = s_ab[1];
          first = false;
        }
        if (ok) {
          const float4 Pn = make_float4(rv.x + beta * pv.x, rv.y + beta * pv.y, rv.z + beta * pv.z, rv.w + beta * pv.w);
          st4(x, g0, make_float4(xv.x + alpha * Pn.x, xv.y + alpha * Pn.y, xv.z + alpha * Pn.z, xv.w + alpha * Pn.w));
        }
      }
      return;
    }
  }
  constexpr int PT = PerThread<T>::value;
  for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * PT) {
    T rv[PT], pv[PT], xv[PT];
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) {
        rv[e] = r[g];
        pv[e] = p[g];
        xv[e] = x[g];
      }
    }
    if (first) {
      cg_scalars<T>(tl, in, sc, ph, s_ab, &s_go);
      if (!s_go) return;
      alpha = s_ab[0];
      beta = s_ab[1];
      first = false;
    }
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
      if (g < end) {
        const T pi = rv[e] + beta * pv[e];
        x[g] = xv[e] + alpha * pi;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_last(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                      InstScal *__restrict__ scal, int ph, unsigned long long *ts,
                                                      const __grid_constant__ CgOne one) {
  const Stamp stamp(ts);
  if (one.on) {
    body_cg_last_in<T>(one_tile(one), one.d, scal[0], ph);
  } else {
    const Tile tl = tiles[blockIdx.x];
    body_cg_last_in<T>(tl, insts[tl.inst], scal[tl.inst], ph);
  }
}

// The first step launch of an iteration (phase 2): beta = 0, so p_0 = r_0 and
// s_0 = w_0 without reading p or s; its own kernel keeps the other steps'
// register allocation.
template <typename T, bool BL = false>
__global__ void __launch_bounds__(kThreads, 3) k_cg_first(const Tile *__restrict__ tiles,
                                                         const InstDev *__restrict__ insts,
                                                         InstScal *__restrict__ scal, int ph, unsigned long long *ts,
                                                         const __grid_constant__ CgOne one) {
  const Stamp stamp(ts);
  if constexpr (BL) {
    if (!one.on && tiles[blockIdx.x].item > 0) return;  // k_cg_step_blur's items
  }
  if (one.on) {
    body_cg_step_in<T, CgDesc, true>(one_tile(one), one.d, scal[0], ph);
  } else {
    const Tile tl = tiles[blockIdx.x];
    body_cg_step_in<T, InstDev, true>(tl, insts[tl.inst], scal[tl.inst], ph);
  }
}

template <typename T, bool BL = false>
__global__ void __launch_bounds__(kThreads, 3) k_cg_step(const Tile *__restrict__ tiles,
                                                         const InstDev *__restrict__ insts,
                                                         InstScal *__restrict__ scal, int ph, unsigned long long *ts,
                                                         const __grid_constant__ CgOne one) {
  const Stamp stamp(ts);
  if constexpr (BL) {
    if (!one.on && tiles[blockIdx.x].item > 0) return;  // k_cg_step_blur's items
  }
  if (one.on)
    body_cg_step_in<T>(one_tile(one), one.d, scal[0], ph);
  else
    cg_step_call<T>(tiles[blockIdx.x], insts, scal, ph);
}

// --------------------------------------------------------------------------
// Instances with a blur block: block work items staged in shared memory.
// The point j of a block item (tz = item rows along z, ta samples along the
// blur axis) is g = start + (j % tz) + (j / tz) st.  The CTA first stages
// the block's values plus a halo of H samples (R for F, 2R for F^T F)
// along the axis and, for an x or y blur, one z row on either side, zero
// outside the grid: every tap of F or F^T F and the z and blur-axis
// neighbours of the 7-point stencil read shared memory.
// --------------------------------------------------------------------------
struct BlurBlk {
  int64_t g0, st;
  int tz, ta, z0, a0, nz, na, R;
};
template <typename D>
__device__ __forceinline__ BlurBlk blur_blk(const D &in, const Tile &tl) {
  BlurBlk b;
  b.g0 = tl.start;
  b.st = in.bl_st;
  b.tz = tl.item;
  b.ta = tl.len / tl.item;
  b.z0 = (int)((uint32_t)tl.start - (uint32_t)in.nz * fdiv((uint32_t)tl.start, in.fz));
  b.a0 = blur_pos(in, tl.start);
  b.nz = in.nz;
  b.na = in.bl_n;
  b.R = in.bl_R;
  return b;
}
// Row pitch of a staged buffer, a compile-time constant of the hot loops
// (the kernels pick the instantiation from the item's z rows): 1 for a z
// blur, else kBlurTZ + 2 (the block's z rows and one halo row either side).
template <int PP> struct BlurPitch {
  static constexpr int P = PP, zo = PP == 1 ? 0 : 1, tz = PP == 1 ? 1 : kBlurTZ;
};
// local point j -> (z row, sample along the axis, grid point); false for
// the slots of a ragged block that fall outside the grid
template <int PP>
__device__ __forceinline__ bool blur_pt(const BlurBlk &b, int j, int &zz, int &aa, int64_t &g) {
  constexpr int tz = BlurPitch<PP>::tz;
  zz = tz == 1 ? 0 : (j & (kBlurTZ - 1));
  aa = tz == 1 ? j : j / kBlurTZ;
  g = b.g0 + zz + (int64_t)aa * b.st;
  return j < tz * b.ta && b.a0 + aa < b.na && (tz == 1 || b.z0 + zz < b.nz);
}
// buf[(zz + zo) + (c + H) P] = f(g of z row zz, offset c along the axis)
// for zz in [-zo, tz + zo), c in [-H, ta + H); 0 outside the grid
template <int PP, typename T, typename F>
__device__ __forceinline__ void blur_stage(const BlurBlk &b, int H, T *buf, F f) {
  using BP = BlurPitch<PP>;
  const int cnt = BP::P * (b.ta + 2 * H);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
    const int c = idx / BP::P - H;
    const int zz = idx - (c + H) * BP::P - BP::zo;
    const int pa = b.a0 + c, pz = b.z0 + zz;
    const bool ok = pa >= 0 && pa < b.na && (BP::tz == 1 || (pz >= 0 && pz < b.nz));
    buf[idx] = ok ? f(b.g0 + zz + (int64_t)c * b.st) : T(0);
  }
}
// the staged value at (zz, aa) for a buffer with halo H
template <int PP, typename T>
__device__ __forceinline__ const T *blur_at(const T *buf, int H, int zz, int aa) {
  return buf + (zz + BlurPitch<PP>::zo) + (aa + H) * BlurPitch<PP>::P;
}
// taps k_0..k_R and autocorrelation a_0..a_2R of the blur table
template <typename T, typename D>
__device__ __forceinline__ void blur_coef(const D &in, T *cf) {
  const T *__restrict__ tab = (const T *)in.bl_w;
  for (int t = threadIdx.x; t < 3 * in.bl_R + 2; t += blockDim.x) cf[t] = tab[t];
}
// (F v) at the staged point p (halo >= R)
template <int PP, typename T>
__device__ __forceinline__ T blur_fwd_buf(const BlurBlk &b, const T *p, const T *k) {
  constexpr int P = BlurPitch<PP>::P;
  T s = k[0] * p[0];
#pragma unroll 4
  for (int t = 1; t <= b.R; ++t) s += k[t] * (p[-t * P] + p[t * P]);
  return s;
}
// (F^T F v) at the staged point p of sample aa (halo 2R).  Row i of F^T F
// is sum_{0 <= j < n} k_|i-j| k_|l-j| at column l.  Summed over every j it
// is the kernel's autocorrelation a_|i-l|; the rows j < 0 are missing only
// where i and l are both below R (the correction E[i][l]), and the rows
// j >= n, by the mirror symmetry j -> n-1-j, only where both are within R
// of the far end (E[n-1-i][n-1-l]).
template <int PP, typename T>
__device__ __forceinline__ T blur_normal_buf(const BlurBlk &b, const T *p, const T *a, const T *__restrict__ E,
                                             int aa) {
  constexpr int P = BlurPitch<PP>::P;
  const int R = b.R, n = b.na, i = b.a0 + aa;
  T s = a[0] * p[0];
#pragma unroll 4
  for (int d = 1; d <= 2 * R; ++d) s += a[d] * (p[-d * P] + p[d * P]);
  const int L = R < n ? R : n;
  if (i < R)
    for (int l = 0; l < L; ++l) s -= E[i * R + l] * p[(l - i) * P];
  if (i >= n - R) {
    const int ii = n - 1 - i;
    for (int l = 0; l < L; ++l) s -= E[ii * R + l] * p[(n - 1 - l - i) * P];
  }
  return s;
}
// 7-point stencil values at g (Nbr convention: a missing neighbour repeats
// the centre): the z and blur-axis neighbours from the staged point p, the
// third axis from v(i)
template <int PP, typename T, typename V>
__device__ __forceinline__ void blur_nbr(const InstDev &in, const GridPos &ps, int64_t g, const T *p, T cv, V v,
                                         Nbr<T> &o) {
  const int64_t sxy = (int64_t)in.nz * in.nx;
  constexpr int P = BlurPitch<PP>::P;
  o.c = cv;
  o.zm = ps.iz > 0 ? p[-1] : cv;
  o.zp = ps.iz < in.nz - 1 ? p[1] : cv;
  if (PP == 1 || in.bl_axis == 2) {
    o.xm = ps.ix > 0 ? v(g - in.nz) : cv;
    o.xp = ps.ix < in.nx - 1 ? v(g + in.nz) : cv;
  } else {
    o.xm = ps.ix > 0 ? p[-P] : cv;
    o.xp = ps.ix < in.nx - 1 ? p[P] : cv;
  }
  if (PP == 1 || in.bl_axis == 1) {
    o.ym = ps.iy > 0 ? v(g - sxy) : cv;
    o.yp = ps.iy < in.ny - 1 ? v(g + sxy) : cv;
  } else {
    o.ym = ps.iy > 0 ? p[-P] : cv;
    o.yp = ps.iy < in.ny - 1 ? p[P] : cv;
  }
}
constexpr int kBlurCoef = 3 * SIP_MAX_BLUR_RADIUS + 2;

// Box kernels (every tap k_0: the paper's motion blur) on x or y blocks:
// F v is k_0 times a window sum, which a thread slides over kBoxRun
// positions along the axis (one add and one subtract per step) instead of
// summing 2R + 1 taps per point.  F^T F v = F (M F v) with M zeroing the
// positions outside the grid (F's rows are the grid's samples), so the
// ends need no correction table.
constexpr int kBoxRun = 8;
constexpr int kBoxU = kBlurTZ * (kBlurTA + 2 * SIP_MAX_BLUR_RADIUS);
constexpr int kBoxO = kBlurTZ * kBlurTA;
// dst(zz, c) = k sum_{|t| <= R} src(zz, c + t) for c in [lo, hi) and every
// z row of the block, src(zz, c) = src[sz + zz + c sp], dst(zz, c) =
// dst[zz + (c - lo) kBlurTZ]; with mask, 0 where c is outside the grid
template <typename T>
__device__ __forceinline__ void box_pass(const BlurBlk &b, const T *src, int sp, int sz, T *dst, int lo, int hi, T k,
                                         bool mask) {
  const int R = b.R, nrun = (hi - lo + kBoxRun - 1) / kBoxRun;
  for (int w = threadIdx.x; w < kBlurTZ * nrun; w += blockDim.x) {
    const int zz = w & (kBlurTZ - 1), c0 = lo + (w / kBlurTZ) * kBoxRun;
    const int c1 = c0 + kBoxRun < hi ? c0 + kBoxRun : hi;
    const T *sr = src + sz + zz;
    T acc = T(0);
    for (int t = -R; t <= R; ++t) acc += sr[(c0 + t) * sp];
    for (int c = c0; c < c1; ++c) {
      if (c > c0) acc += sr[(c + R) * sp] - sr[(c - R - 1) * sp];
      const int pa = b.a0 + c;
      dst[zz + (c - lo) * kBlurTZ] = (!mask || (pa >= 0 && pa < b.na)) ? k * acc : T(0);
    }
  }
}
// F^T F v at the block's points into ob(zz, aa) = ob[zz + aa kBlurTZ],
// from v staged with halo 2R (pitch kBlurTZ + 2); ub holds M F v
template <typename T>
__device__ __forceinline__ void box_normal(const BlurBlk &b, const T *buf, T *ub, T *ob, T k) {
  constexpr int P = kBlurTZ + 2;
  const int R = b.R;
  box_pass(b, buf, P, 1 + 2 * R * P, ub, -R, b.ta + R, k, true);
  __syncthreads();
  box_pass(b, ub, kBlurTZ, R * kBlurTZ, ob, 0, b.ta, k, false);
  __syncthreads();
}
// F v at the block's points into ob, from v staged with halo R
template <typename T>
__device__ __forceinline__ void box_fwd(const BlurBlk &b, const T *buf, T *ob, T k) {
  constexpr int P = kBlurTZ + 2;
  box_pass(b, buf, P, 1 + b.R * P, ob, 0, b.ta, k, false);
  __syncthreads();
}

// The blur block's part of the x-step's right-hand side and warm residual,
// t = F^T (rho_F y_F + v_F) - rho_F F^T F x, into the instance's F x
// scratch (free between the set pass and the next right-hand side); the
// right-hand side launch adds it at every grid point.
template <typename T, int PP>
__device__ __forceinline__ void blur_rhs_p(const Tile &tl, const InstDev &in, const InstScal &sc, T *buf, T *cf,
                                           T *ub, T *ob) {
  constexpr int NE = kBlurLen / kThreads;
  const bool box = PP != 1 && in.bl_box;
  const BlurBlk b = blur_blk(in, tl);
  const T *__restrict__ x = (const T *)in.x;
  T *__restrict__ t = (T *)in.bl_s;
  const int64_t yo = in.blk[in.bl_blk].yoff;
  const T *__restrict__ yF = (const T *)in.y + yo;
  const T *__restrict__ vF = (const T *)in.v + yo;
  const T rhoF = SV<T>::blk(sc, in.bl_blk, BF_RHO);
  blur_coef<T>(in, cf);
  blur_stage<PP>(b, b.R, buf, [&](int64_t q) { return rhoF * yF[q] + vF[q]; });
  __syncthreads();
  if constexpr (PP != 1) {
    if (box) box_fwd(b, buf, ob, cf[0]);
  }
  T tv[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int zz, aa;
    int64_t g;
    tv[e] = T(0);
    if (blur_pt<PP>(b, threadIdx.x + e * kThreads, zz, aa, g))
      tv[e] = box ? ob[zz + aa * kBlurTZ] : blur_fwd_buf<PP>(b, blur_at<PP>(buf, b.R, zz, aa), cf);
  }
  __syncthreads();
  blur_stage<PP>(b, 2 * b.R, buf, [&](int64_t q) { return x[q]; });
  __syncthreads();
  if constexpr (PP != 1) {
    if (box) box_normal(b, buf, ub, ob, cf[0]);
  }
  const T *__restrict__ E = (const T *)in.bl_w + 3 * b.R + 2;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int zz, aa;
    int64_t g;
    if (blur_pt<PP>(b, threadIdx.x + e * kThreads, zz, aa, g))
      t[g] = tv[e] - rhoF * (box ? ob[zz + aa * kBlurTZ]
                                 : blur_normal_buf<PP>(b, blur_at<PP>(buf, 2 * b.R, zz, aa), cf + b.R + 1, E, aa));
  }
}
template <typename T>
__global__ void __launch_bounds__(kThreads) k_blur_rhs(const Tile *__restrict__ tiles,
                                                      const InstDev *__restrict__ insts,
                                                      const InstScal *__restrict__ scal, unsigned long long *ts) {
  const Stamp stamp(ts);
  __shared__ T buf[kBlurBuf];
  __shared__ T cf[kBlurCoef];
  __shared__ T ub[kBoxU];
  __shared__ T ob[kBoxO];
  const Tile tl = tiles[blockIdx.x];
  if (tl.item <= 0) return;
  const InstDev &in = insts[tl.inst];
  const InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  if (tl.item == 1)
    blur_rhs_p<T, 1>(tl, in, sc, buf, cf, ub, ob);
  else
    blur_rhs_p<T, kBlurTZ + 2>(tl, in, sc, buf, cf, ub, ob);
}

// w_0 = C r_0 of a blur block item
template <typename T, int PP>
__device__ __forceinline__ void cg_w0_blur_p(const Tile &tl, const InstDev &in, InstScal &sc, T *buf, T *cf, T *ub,
                                             T *ob) {
  using A = typename AccOf<T>::type;
  const bool box = PP != 1 && in.bl_box;
  const BlurBlk b = blur_blk(in, tl);
  const int H = 2 * b.R;
  const T *__restrict__ r = (const T *)in.cr[0];
  T *__restrict__ w = (T *)in.cw[0];
  blur_coef<T>(in, cf);
  blur_stage<PP>(b, H, buf, [&](int64_t q) { return r[q]; });
  __syncthreads();
  if constexpr (PP != 1) {
    if (box) box_normal(b, buf, ub, ob, cf[0]);
  }
  CSys<T> C;
  C.load(sc);
  const T rhoF = SV<T>::blk(sc, in.bl_blk, BF_RHO);
  const T *__restrict__ E = (const T *)in.bl_w + 3 * b.R + 2;
  A a0 = A(0);
  for (int j = threadIdx.x; j < tl.len; j += kThreads) {
    int zz, aa;
    int64_t g;
    if (!blur_pt<PP>(b, j, zz, aa, g)) continue;
    const T *pc = blur_at<PP>(buf, H, zz, aa);
    Nbr<T> rn;
    blur_nbr<PP>(in, grid_pos(in, g), g, pc, pc[0], [&](int64_t i) { return r[i]; }, rn);
    const T band = box ? ob[zz + aa * kBlurTZ] : blur_normal_buf<PP>(b, pc, cf + b.R + 1, E, aa);
    const T wg = apply_c(C, rn) + rhoF * band;
    w[g] = wg;
    a0 += (A)wg * (A)rn.c;
  }
  A acc[1] = {a0};
  block_sum<1>(acc);
  if (threadIdx.x == 0) cg_part<A>(in, 2, 0)[tl.seq] = acc[0];  // delta_0 = r_0^T C r_0
}
template <typename T>
__device__ void body_cg_w0_blur(const Tile &tl, const InstDev &in, InstScal &sc) {
  __shared__ T buf[kBlurBuf];
  __shared__ T cf[kBlurCoef];
  __shared__ T ub[kBoxU];
  __shared__ T ob[kBoxO];
  if (sc.done) return;
  if (tl.item == 1)
    cg_w0_blur_p<T, 1>(tl, in, sc, buf, cf, ub, ob);
  else
    cg_w0_blur_p<T, kBlurTZ + 2>(tl, in, sc, buf, cf, ub, ob);
}

// One CG step of a blur block item: the general step's arithmetic, with
// r_{i+1} = r_i - alpha (w_i + beta s_{i-1}) staged over the block and its
// halo for the F^T F band and the stencil neighbours
template <typename T, int PP>
__device__ __forceinline__ void cg_step_blur_p(const Tile &tl, const InstDev &in, InstScal &sc, int ph, T *buf,
                                               T *cf, T *ub, T *ob, T *s_ab, int *s_go) {
  using A = typename AccOf<T>::type;
  const bool box = PP != 1 && in.bl_box;
  const int c = ph & 1, n = c ^ 1;
  const T *__restrict__ r = (const T *)in.cr[c];
  const T *__restrict__ w = (const T *)in.cw[c];
  const T *__restrict__ sp = (const T *)in.cs[c];  // s_{i-1}
  T *__restrict__ rn_ = (T *)in.cr[n];
  T *__restrict__ wn_ = (T *)in.cw[n];
  T *__restrict__ sn_ = (T *)in.cs[n];             // s_i
  T *__restrict__ p = (T *)in.cp;
  T *__restrict__ x = (T *)in.x;
  // the item's p and x, in flight while the scalars and the stage arrive
  constexpr int NE = kBlurLen / kThreads;
  const BlurBlk b = blur_blk(in, tl);
  T pv[NE], xv[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int zz, aa;
    int64_t g;
    pv[e] = xv[e] = T(0);
    if (blur_pt<PP>(b, threadIdx.x + e * kThreads, zz, aa, g)) {
      pv[e] = p[g];
      xv[e] = x[g];
    }
  }
  cg_scalars<T>(tl, in, sc, ph, s_ab, s_go);
  if (!*s_go) return;
  const T alpha = s_ab[0], beta = s_ab[1];
  const int H = 2 * b.R;
  auto rnew_at = [&](int64_t q) { return r[q] - alpha * (w[q] + beta * sp[q]); };
  blur_coef<T>(in, cf);
  blur_stage<PP>(b, H, buf, rnew_at);
  __syncthreads();
  if constexpr (PP != 1) {
    if (box) box_normal(b, buf, ub, ob, cf[0]);
  }
  CSys<T> C;
  C.load(sc);
  const T rhoF = SV<T>::blk(sc, in.bl_blk, BF_RHO);
  const T *__restrict__ E = (const T *)in.bl_w + 3 * b.R + 2;
  A ag = A(0), ad = A(0);
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    int zz, aa;
    int64_t g;
    if (!blur_pt<PP>(b, threadIdx.x + e * kThreads, zz, aa, g)) continue;
    const T rv = r[g], wv = w[g], sv = sp[g];
    const T *pc = blur_at<PP>(buf, H, zz, aa);
    const T s_c = wv + beta * sv;
    const T rc = rv - alpha * s_c;
    Nbr<T> rnew;
    blur_nbr<PP>(in, grid_pos(in, g), g, pc, rc, rnew_at, rnew);
    const T pi = rv + beta * pv[e];
    p[g] = pi;
    x[g] = xv[e] + alpha * pi;
    sn_[g] = s_c;
    rn_[g] = rc;
    const T band = box ? ob[zz + aa * kBlurTZ] : blur_normal_buf<PP>(b, pc, cf + b.R + 1, E, aa);
    const T wnew = apply_c(C, rnew) + rhoF * band;
    wn_[g] = wnew;
    ag += (A)rc * (A)rc;
    ad += (A)wnew * (A)rc;
  }
  A acc[2] = {ag, ad};
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    const int slot = 1 + (ph & 1);
    cg_part<A>(in, slot, 0)[tl.seq] = acc[0];
    cg_part<A>(in, slot, 1)[tl.seq] = acc[1];
  }
}
template <typename T>
__device__ void body_cg_step_blur(const Tile &tl, const InstDev &in, InstScal &sc, int ph) {
  __shared__ T buf[kBlurBuf];
  __shared__ T cf[kBlurCoef];
  __shared__ T ub[kBoxU];
  __shared__ T ob[kBoxO];
  __shared__ T s_ab[2];
  __shared__ int s_go;
  if (tl.item == 1)
    cg_step_blur_p<T, 1>(tl, in, sc, ph, buf, cf, ub, ob, s_ab, &s_go);
  else
    cg_step_blur_p<T, kBlurTZ + 2>(tl, in, sc, ph, buf, cf, ub, ob, s_ab, &s_go);
}

// The CG step of the blur block items, a kernel of its own so that its
// register budget (and so its residency: the step is latency-bound) is not
// the general step's
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) k_cg_step_blur(const Tile *__restrict__ tiles,
                                                              const InstDev *__restrict__ insts,
                                                              InstScal *__restrict__ scal, int ph,
                                                              unsigned long long *ts) {
  const Stamp stamp(ts);
  const Tile tl = tiles[blockIdx.x];
  if (tl.item <= 0) return;  // the general step's items
  body_cg_step_blur<T>(tl, insts[tl.inst], scal[tl.inst], ph);
}

// s = F x of every blur block item, for the set pass
template <typename T, int PP>
__device__ __forceinline__ void blur_fwd_p(const Tile &tl, const InstDev &in, T *buf, T *cf, T *ob) {
  const bool box = PP != 1 && in.bl_box;
  const BlurBlk b = blur_blk(in, tl);
  const T *__restrict__ x = (const T *)in.x;
  T *__restrict__ sF = (T *)in.bl_s;
  blur_coef<T>(in, cf);
  blur_stage<PP>(b, b.R, buf, [&](int64_t q) { return x[q]; });
  __syncthreads();
  if constexpr (PP != 1) {
    if (box) box_fwd(b, buf, ob, cf[0]);
  }
  for (int j = threadIdx.x; j < tl.len; j += kThreads) {
    int zz, aa;
    int64_t g;
    if (blur_pt<PP>(b, j, zz, aa, g))
      sF[g] = box ? ob[zz + aa * kBlurTZ] : blur_fwd_buf<PP>(b, blur_at<PP>(buf, b.R, zz, aa), cf);
  }
}
template <typename T>
__global__ void __launch_bounds__(kThreads) k_blur_fwd(const Tile *__restrict__ tiles,
                                                      const InstDev *__restrict__ insts,
                                                      const InstScal *__restrict__ scal, unsigned long long *ts) {
  const Stamp stamp(ts);
  __shared__ T buf[kBlurBuf];
  __shared__ T cf[kBlurCoef];
  __shared__ T ob[kBoxO];
  const Tile tl = tiles[blockIdx.x];
  if (tl.item <= 0) return;
  const InstDev &in = insts[tl.inst];
  if (scal[tl.inst].done) return;
  if (tl.item == 1)
    blur_fwd_p<T, 1>(tl, in, buf, cf, ob);
  else
    blur_fwd_p<T, kBlurTZ + 2>(tl, in, buf, cf, ob);
}

// --------------------------------------------------------------------------
// Set pass: relaxation, prox input, point-wise prox, dual update, stopping
// and adapt inner products (Algorithm PARSDMM FOR-body; Algorithm
// adapt-rho-gamma; Eqs. feas_stop, obj_stop)
// --------------------------------------------------------------------------
template <typename T>
__device__ void setpass_ring(const Tile &tl, const InstDev &in, InstScal &sc, int k, bool chk) {
  SIP_STEP_CONSTANTS;
  using A = typename AccOf<T>::type;
  // x^k against the stored x^{k-1} .. x^{k-s} (Eq. obj_stop), then store x^k.
  const T *__restrict__ x = (const T *)in.x;
  T *__restrict__ ring = (T *)in.ring;
  const int H = in.hist;
  const int jmax = k < H ? k : H;
  const int64_t N = in.N;
  const int64_t wslot = (int64_t)(k % H) * N;
  const int64_t end = tl.start + tl.len;
  A acc[kMaxHist + 1];
#pragma unroll
  for (int j = 0; j <= kMaxHist; ++j) acc[j] = A(0);
  bool vec = false;
  if constexpr (sizeof(T) == 4)
    vec = (N & 3) == 0 && (tl.start & 3) == 0 && (((uintptr_t)x | (uintptr_t)ring) & 15) == 0;
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      // 16-byte accesses: 4 consecutive samples per thread
      for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * 4) {
        const int64_t g0 = base + (int64_t)threadIdx.x * 4;
        if (g0 >= end) continue;
        const float4 X = ld4(x, g0);  // N % 4 == 0: no partial group
        if (chk) {
#pragma unroll
          for (int j = 1; j <= kMaxHist; ++j) {
            if (j <= jmax) {
              const float4 Hv = ld4(ring, (int64_t)((k - j) % H) * N + g0);
              const A d0 = (A)X.x - (A)Hv.x, d1 = (A)X.y - (A)Hv.y, d2 = (A)X.z - (A)Hv.z, d3 = (A)X.w - (A)Hv.w;
              acc[j] += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            }
          }
          acc[0] += (A)X.x * (A)X.x + (A)X.y * (A)X.y + (A)X.z * (A)X.z + (A)X.w * (A)X.w;
        }
        st4(ring, wslot + g0, X);
      }
    }
  } else {
    for (int64_t base = tl.start; base < end; base += SUB) {
      T xv[PT];
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
        if (g < end) xv[e] = x[g];
      }
      if (chk) {
#pragma unroll
        for (int j = 1; j <= kMaxHist; ++j) {
          if (j <= jmax) {
            const int64_t so = (int64_t)((k - j) % H) * N;
            T hv[PT];
#pragma unroll
            for (int e = 0; e < PT; ++e) {
              const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
              if (g < end) hv[e] = ring[so + g];
            }
#pragma unroll
            for (int e = 0; e < PT; ++e) {
              const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
              if (g < end) {
                const A d = (A)xv[e] - (A)hv[e];
                acc[j] += d * d;
              }
            }
          }
        }
      }
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t g = base + threadIdx.x + (int64_t)e * kThreads;
        if (g < end) {
          if (chk) acc[0] += (A)xv[e] * (A)xv[e];
          ring[wslot + g] = xv[e];
        }
      }
    }
  }
  if (chk) {
    block_sum<kMaxHist + 1>(acc);
    if (threadIdx.x == 0)
      for (int j = 0; j <= jmax; ++j) atomicAdd(&sc.acc_ring[j], (double)acc[j]);
  }
}

// The block's per-iteration scalars, in the storage type.
template <typename T>
struct SetpassScal {
  T rho, irho, gam, one_m_gam, inv1p, lo, hi, ih;
  int type, kind;
  bool pointwise, ad, ad_dots, chk;
  bool centered;  // l2 data fit: the row's observed value comes as `lo` (NaN: unobserved)
};

// What one row stores: the dual update's y and v (point-wise sets) or the
// prox input w (sets projected after a selection), and the adapt copies.
template <typename T>
struct RowOut {
  T yn, vn, w, vh;
};

// One row of the set pass: relaxation, prox input, point-wise prox and dual
// update, adapt-rho-gamma and feasibility partial sums (Algorithm PARSDMM
// FOR-body; Algorithm adapt-rho-gamma; Eq. feas_stop).
// Partials: 0..5 adapt dots, 6 feasD2, 7 s2, 8 s1, 9 wnorm.
// PW: 0 any block type (decided per row from q), 1 bounds, 2 the identity
// block's distance prox (the block type fixed at compile time)
template <int PW = 0, typename T, typename A>
__device__ __forceinline__ RowOut<T> setpass_row(const SetpassScal<T> &q, T s, T y0, T v0, T mg, T ks, T kvh, T ky,
                                                 T kv, T lo, T hi, A (&acc)[10]) {
  RowOut<T> o;
  const T xbar = q.gam * s + q.one_m_gam * y0;
  o.w = xbar - v0 * q.irho;
  o.vh = T(0);
  if (q.ad) {
    // vhat^{k+1} = v^k + rho (y^k - s^{k+1}); dh = s - s^{k0}; dvh = vhat - vhat^{k0}
    o.vh = v0 + q.rho * (y0 - s);
    if (q.ad_dots) {
      const A dh = (A)s - (A)ks;
      const A dvh = (A)o.vh - (A)kvh;
      acc[0] += dh * dvh;
      acc[1] += dh * dh;
      acc[2] += dvh * dvh;
    }
  }
  const bool pointwise = PW ? true : q.pointwise;
  const bool bounds = PW ? PW == 1 : q.type == BT_BOUNDS;
  if (pointwise) {
    o.yn = bounds ? fmin(fmax(o.w, lo), hi) : (mg + q.rho * o.w) * q.inv1p;  // Eq. prox_sq_dist
    o.vn = v0 + q.rho * (o.yn - xbar);
    if (q.ad_dots) {
      const A dg = (A)ky - (A)o.yn;
      const A dv = (A)o.vn - (A)kv;
      acc[3] += dg * dv;
      acc[4] += dg * dg;
      acc[5] += dv * dv;
    }
    if (q.chk && bounds) {
      const A d = (A)s - (A)fmin(fmax(s, lo), hi);
      acc[6] += d * d;
      acc[7] += (A)s * (A)s;
    }
  } else {
    o.yn = o.vn = T(0);
    if (q.centered) {  // ||w - d|| and ||s - d|| over the observed rows
      if (!isnan(lo)) {
        const A r = (A)o.w - (A)lo;
        acc[9] += r * r;
        if (q.chk) {
          const A rs = (A)s - (A)lo;
          acc[6] += rs * rs;
        }
      }
    } else if (q.type == BT_L2 || q.type == BT_ANNULUS) {
      acc[9] += (A)o.w * (A)o.w;
    }
    if (q.type == BT_L1) acc[9] += fabs((A)o.w);
    if (q.chk) {
      acc[7] += (A)s * (A)s;
      if (q.type == BT_L1) acc[8] += fabs((A)s);
    }
  }
  return o;
}

template <typename T, bool BL = false>
__device__ void setpass_block(const Tile &tl, const InstDev &in, InstScal &sc, const SegDev &sg, int k, bool ad,
                              bool ad_dots, bool chk, JobScal *__restrict__ jscal,
                              const JobDev *__restrict__ jobs) {
  SIP_STEP_CONSTANTS;
  using A = typename AccOf<T>::type;
  const int b = sg.block;
  const BlockDev &bd = in.blk[b];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= sg.len && sg.row0 + sg.len <= bd.M, 4u,
                 sg.row0 + tl.start + tl.len);
  SetpassScal<T> q;
  q.rho = SV<T>::blk(sc, b, BF_RHO);
  q.irho = SV<T>::blk(sc, b, BF_IRHO);
  q.gam = SV<T>::blk(sc, b, BF_GAMMA);
  q.one_m_gam = SV<T>::blk(sc, b, BF_OMG);
  q.inv1p = SV<T>::blk(sc, b, BF_INV1P);
  q.lo = (T)bd.lo;
  q.hi = (T)bd.hi;
  q.ih = seg_ih<T>(in, sg.kind);
  q.kind = sg.kind;
  q.type = bd.type;
  q.pointwise = bd.type == BT_BOUNDS || bd.type == BT_DIST;
  q.centered = bd.type == BT_L2 && bd.bv_lo >= 0;
  q.ad = ad;
  q.ad_dots = ad_dots;
  q.chk = chk;
  const int kind = sg.kind, type = bd.type;
  const bool pointwise = q.pointwise;
  const bool store_s = chk && bd.soff >= 0;  // selections and per-line sets project s
  const T *__restrict__ x = (const T *)in.x;
  T *__restrict__ y = (T *)in.y + bd.yoff + sg.row0;
  T *__restrict__ v = (T *)in.v + bd.yoff + sg.row0;
  T *__restrict__ wbuf = (T *)in.w + bd.woff + sg.row0;
  T *__restrict__ sbuf = (T *)in.s + bd.soff + sg.row0;
  T *__restrict__ k0s = (T *)in.k0s + bd.yoff + sg.row0;
  T *__restrict__ k0vh = (T *)in.k0vh + bd.yoff + sg.row0;
  T *__restrict__ k0y = (T *)in.k0y + bd.yoff + sg.row0;
  T *__restrict__ k0v = (T *)in.k0v + bd.yoff + sg.row0;
  const T *__restrict__ m = (const T *)in.m;
  // per-entry bounds (point-wise data fit), else the scalars q.lo, q.hi
  const T *__restrict__ blo = bd.bv_lo >= 0 ? (const T *)in.bvec + bd.bv_lo + sg.row0 : nullptr;
  const T *__restrict__ bhi = bd.bv_hi >= 0 ? (const T *)in.bvec + bd.bv_hi + sg.row0 : nullptr;
  const int64_t end = tl.start + tl.len;
  A acc[10];
#pragma unroll
  for (int j = 0; j < 10; ++j) acc[j] = A(0);
  // top-k window (card w-job): count the keys above it, store the keys in it
  using KT = KeyOf<T>;
  using K = typename KT::K;
  bool win = false;
  K wlo = 0, whi = 0;
  K *__restrict__ cand = nullptr;
  uint32_t *wn = nullptr;
  uint32_t above = 0;
  if (type == BT_CARD && bd.job_w >= 0) {
    JobScal &js = jscal[bd.job_w];
    if (js.win_on) {
      win = true;
      wlo = KT::key((T)js.win_lo);
      whi = KT::key((T)js.win_hi);
      cand = (K *)jobs[bd.job_w].cand;
      wn = &js.win_n;
    }
  }
  // called by every active lane of the warp (warp-aggregated slot claims)
  auto classify = [&](T wv, bool valid) {
    const K key = KT::key(wv);
    if (valid && key > whi) ++above;
    const bool inw = valid && key >= wlo && key <= whi;
    const unsigned am = __activemask();
    const unsigned bal = __ballot_sync(am, inw);
    if (bal) {
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(bal) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(wn, (uint32_t)__popc(bal));
      base = __shfl_sync(am, base, leader);
      if (inw) {
        const uint32_t pos = base + (uint32_t)__popc(bal & ((1u << lane) - 1u));
        if (pos < (uint32_t)kWinCap) cand[pos] = key;
      }
    }
  };
  // s^{k0} = A x^{k0} of the last adapt iteration, from x^{k0} in the x
  // history ring (k0ring) or from the stored copy k0s
  const bool k0ring = in.k0_ring != 0;
  // (the slot of iteration k - adapt_every, taken modulo the ring length
  // also when that iteration precedes this projection: a warm start that
  // carries the adapt state puts x^{k0} there)
  const T *__restrict__ xk0 =
      (k0ring && ad_dots)
          ? (const T *)in.ring + (int64_t)(((k - in.adapt_every) % in.hist + in.hist) % in.hist) * in.N
          : nullptr;
  // x gathers of one row: s = A x (Eq. FD_mat), m at the base sample and,
  // from the ring, s^{k0}
  auto gather = [&](int64_t row, T &sv, T &mv, T &kv0) {
    int64_t off;
    int64_t g = seg_base(in, kind, row, off);
    if (!SIP_GUARD_IDX(in.err, g >= 0 && g + off >= 0 && g < in.N && g + off < in.N, 5u, g)) g = off = 0;
    const T x0 = x[g];
    sv = kind == SEG_I ? x0 : (x[g + off] - x0) * q.ih;
    mv = type == BT_DIST ? m[g] : T(0);
    if (xk0) {
      const T z0 = xk0[g];
      kv0 = kind == SEG_I ? z0 : (xk0[g + off] - z0) * q.ih;
    }
    if constexpr (BL) {
      // s = F x, written by the blur kernel before the set pass (blur
      // instances keep s^{k0} in k0s: no x-history gathers)
      if (kind == SEG_BLUR) sv = ((const T *)in.bl_s)[g];
    }
  };
  bool vec = false;
  if constexpr (sizeof(T) == 4) {
    // 16-byte accesses to the row arrays when they all start on a 16-byte
    // boundary at this work item
    uintptr_t al = (uintptr_t)(y + tl.start) | (uintptr_t)(v + tl.start);
    if (ad) al |= (uintptr_t)(k0vh + tl.start);
    if (ad && !k0ring) al |= (uintptr_t)(k0s + tl.start);
    if (ad && pointwise) al |= (uintptr_t)(k0y + tl.start) | (uintptr_t)(k0v + tl.start);
    if (!pointwise) al |= (uintptr_t)(wbuf + tl.start);
    if (store_s) al |= (uintptr_t)(sbuf + tl.start);
    vec = (al & 15) == 0 && !blo;  // per-entry bounds take the scalar path
  }
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      // the block type of the rows' prox, fixed for the whole work item
      const int pwk = type == BT_BOUNDS ? 1 : (type == BT_DIST ? 2 : 0);
      // grouped x gathers of four rows (no blur segment): 1 = identity rows
      // or 2D x-difference rows with 16-byte aligned x (and m, x^{k0}) and
      // n_z % 4 == 0; 2 = z-difference rows; 0 = row by row
      int xfast = 0;
      if (kind == SEG_I || (kind == SEG_DX && in.ny == 1 && (in.nz & 3) == 0)) {
        uintptr_t xa = (uintptr_t)x;
        if (type == BT_DIST) xa |= (uintptr_t)m;
        if (xk0) xa |= (uintptr_t)xk0;
        if ((xa & 15) == 0) xfast = 1;
      } else if (kind == SEG_DZ) {
        xfast = 2;
      }
      for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * 4) {
        const int64_t r0 = base + (int64_t)threadIdx.x * 4;
        if (r0 >= end) continue;
        const bool full = r0 + 4 <= end;
        float4 Y, V, KS = make_float4(0.f, 0.f, 0.f, 0.f), KVH = KS, KY = KS, KV = KS;
        auto ld = [&](const float *p) {
          if (full) return ld4(p, r0);
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int c = 0; c < 4; ++c)
            if (r0 + c < end) vset(t, c, p[r0 + c]);
          return t;
        };
        auto st = [&](float *p, const float4 &t) {
          if (full) {
            st4(p, r0, t);
          } else {
            for (int c = 0; c < 4; ++c)
              if (r0 + c < end) p[r0 + c] = vat(t, c);
          }
        };
        Y = ld(y);
        V = ld(v);
        if (ad_dots) {
          if (!k0ring) KS = ld(k0s);
          KVH = ld(k0vh);
          if (pointwise) {
            KY = ld(k0y);
            KV = ld(k0v);
          }
        }
        float sv[4], mv[4], kr[4];
        if (full && xfast == 1 &&
            SIP_GUARD_IDX(in.err, r0 >= 0 && r0 + 4 + (kind == SEG_DX ? in.nz : 0) <= in.N, 6u, r0)) {
          // identity rows (row = grid point) and 2D x-difference rows (row =
          // grid point, neighbour nz further): 16-byte loads of x
          const float4 xa = ld4(x, r0);
          float4 sa = xa;
          if (kind == SEG_DX) {
            const float4 xb = ld4(x, r0 + in.nz);
            sa = make_float4((xb.x - xa.x) * q.ih, (xb.y - xa.y) * q.ih, (xb.z - xa.z) * q.ih, (xb.w - xa.w) * q.ih);
          }
          float4 ma = make_float4(0.f, 0.f, 0.f, 0.f), ka = ma;
          if (type == BT_DIST) ma = ld4(m, r0);
          if (xk0) {
            const float4 za = ld4(xk0, r0);
            ka = za;
            if (kind == SEG_DX) {
              const float4 zb = ld4(xk0, r0 + in.nz);
              ka = make_float4((zb.x - za.x) * q.ih, (zb.y - za.y) * q.ih, (zb.z - za.z) * q.ih,
                               (zb.w - za.w) * q.ih);
            }
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            sv[c] = vat(sa, c);
            mv[c] = vat(ma, c);
            kr[c] = vat(ka, c);
          }
        } else if (full && xfast == 2) {
          // z-difference rows: one division for the four rows; a row past
          // the end of its column moves on to the next column (grid point
          // = row + column index)
          const uint32_t t = fdiv((uint32_t)r0, in.fzm);
          const int64_t iz0 = r0 - (int64_t)t * (in.nz - 1);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            int64_t g = r0 + c + t + (iz0 + c >= in.nz - 1 ? 1 : 0);
            if (!SIP_GUARD_IDX(in.err, g >= 0 && g + 1 < in.N, 6u, g)) g = 0;
            sv[c] = (x[g + 1] - x[g]) * q.ih;
            mv[c] = 0.f;
            kr[c] = xk0 ? (xk0[g + 1] - xk0[g]) * q.ih : 0.f;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            sv[c] = mv[c] = kr[c] = 0.f;
            if (r0 + c < end) gather(r0 + c, sv[c], mv[c], kr[c]);
          }
        }
        if (xk0) KS = make_float4(kr[0], kr[1], kr[2], kr[3]);
        float4 YN, VN, W, VH;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          RowOut<float> o;
          if (r0 + c < end) {
            if (pwk == 1)
              o = setpass_row<1>(q, sv[c], vat(Y, c), vat(V, c), mv[c], vat(KS, c), vat(KVH, c), vat(KY, c),
                                 vat(KV, c), q.lo, q.hi, acc);
            else if (pwk == 2)
              o = setpass_row<2>(q, sv[c], vat(Y, c), vat(V, c), mv[c], vat(KS, c), vat(KVH, c), vat(KY, c),
                                 vat(KV, c), q.lo, q.hi, acc);
            else
              o = setpass_row<0>(q, sv[c], vat(Y, c), vat(V, c), mv[c], vat(KS, c), vat(KVH, c), vat(KY, c),
                                 vat(KV, c), q.lo, q.hi, acc);
          } else {
            o.yn = o.vn = o.w = o.vh = 0.f;
          }
          if (win) classify(o.w, r0 + c < end);
          vset(YN, c, o.yn);
          vset(VN, c, o.vn);
          vset(W, c, o.w);
          vset(VH, c, o.vh);
        }
        if (ad) {
          if (!k0ring) st(k0s, make_float4(sv[0], sv[1], sv[2], sv[3]));
          st(k0vh, VH);
        }
        if (pointwise) {
          if (in.bf16) {
            YN = rbf4(YN);
            VN = rbf4(VN);
          }
          st(y, YN);
          st(v, VN);
          if (ad) {
            st(k0y, YN);
            st(k0v, VN);
          }
        } else {
          st(wbuf, W);
          if (store_s) st(sbuf, make_float4(sv[0], sv[1], sv[2], sv[3]));
        }
      }
    }
  } else {
    for (int64_t base = tl.start; base < end; base += SUB) {
      T sv[PT], mg[PT], y0[PT], v0[PT];
      T ks[PT], kvh[PT], ky[PT], kv[PT];
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
        ks[e] = kvh[e] = ky[e] = kv[e] = T(0);
        if (row < end) {
          gather(row, sv[e], mg[e], ks[e]);
          y0[e] = y[row];
          v0[e] = v[row];
          if (ad_dots) {
            if (!k0ring) ks[e] = k0s[row];
            kvh[e] = k0vh[row];
            if (pointwise) {
              ky[e] = k0y[row];
              kv[e] = k0v[row];
            }
          }
        }
      }
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
        if (row >= end) continue;
        const RowOut<T> o = setpass_row(q, sv[e], y0[e], v0[e], mg[e], ks[e], kvh[e], ky[e], kv[e],
                                        blo ? blo[row] : q.lo, bhi ? bhi[row] : q.hi, acc);
        if (win) classify(o.w, true);
        if (ad) {
          if (!k0ring) k0s[row] = sv[e];
          k0vh[row] = o.vh;
        }
        if (pointwise) {
          const T yst = in.bf16 ? rbf(o.yn) : o.yn, vst = in.bf16 ? rbf(o.vn) : o.vn;
          y[row] = yst;
          v[row] = vst;
          if (ad) {
            k0y[row] = yst;
            k0v[row] = vst;
          }
        } else {
          wbuf[row] = o.w;
          if (store_s) sbuf[row] = sv[e];
        }
      }
    }
  }
  // CTA sums (in the accumulator type) of only the quantities this
  // iteration uses; binary64 across CTAs
  double *a = sc.acc[b];
  if (ad_dots) {
    A d6[6] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5]};
    block_sum<6>(d6);
    if (threadIdx.x == 0) {
      atomicAdd(&a[A_HV], (double)d6[0]);
      atomicAdd(&a[A_HH], (double)d6[1]);
      atomicAdd(&a[A_VHVH], (double)d6[2]);
      if (pointwise) {
        atomicAdd(&a[A_GV], (double)d6[3]);
        atomicAdd(&a[A_GG], (double)d6[4]);
        atomicAdd(&a[A_VV], (double)d6[5]);
      }
    }
  }
  if (chk && type != BT_DIST) {
    A d3[3] = {acc[6], acc[7], acc[8]};
    block_sum<3>(d3);
    if (threadIdx.x == 0) {
      if (type == BT_BOUNDS || q.centered) atomicAdd(&a[A_FEAS_D2], (double)d3[0]);
      atomicAdd(&a[A_S2], (double)d3[1]);
      if (type == BT_L1) atomicAdd(&a[A_S1], (double)d3[2]);
    }
  }
  if (type == BT_L1 || type == BT_L2 || type == BT_ANNULUS) {
    A d1[1] = {acc[9]};
    block_sum<1>(d1);
    if (threadIdx.x == 0) atomicAdd(&a[A_WNORM], (double)d1[0]);
  }
  if (win) {
    __shared__ uint32_t s_above;
    if (threadIdx.x == 0) s_above = 0;
    __syncthreads();
    const uint32_t wa = __reduce_add_sync(0xffffffffu, above);
    if ((threadIdx.x & 31) == 0 && wa) atomicAdd(&s_above, wa);
    __syncthreads();
    if (threadIdx.x == 0 && s_above)
      atomicAdd((unsigned long long *)&jscal[bd.job_w].win_above, (unsigned long long)s_above);
  }
}

template <typename T, bool BL = false>
__device__ __forceinline__ void body_setpass(const Tile &tl, const InstDev *__restrict__ insts,
                                                      InstScal *__restrict__ scal, JobScal *__restrict__ jscal,
                                                      const JobDev *__restrict__ jobs) {
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  const int k = sc.k;
  const bool ad = adapt_iter(in, k);
  const bool ad_dots = ad && sc.have_k0;
  const bool chk = check_iter(in, k);
  const SegDev sg = in.seg[tl.item];
  if (sg.kind == SEG_RING)
    setpass_ring<T>(tl, in, sc, k, chk);
  else
    setpass_block<T, BL>(tl, in, sc, sg, k, ad, ad_dots, chk, jscal, jobs);

  // The last CTA of the instance resolves the l2 scales and arms the
  // selection jobs of this iteration, one block per lane of warp 0.
  __shared__ bool last;
  if (threadIdx.x == 0) last = arrive_last(&sc.cnt_set, (uint32_t)in.nt_set);
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  const int b = threadIdx.x;
  if (b >= in.nb) return;
  const BlockDev &bd = in.blk[b];
  const double *a = sc.acc[b];
  if (bd.type == BT_L2) {
    const double nrm = sqrt(ldv(&a[A_WNORM]));
    const double sg2 = sc.sigma[b];
    sc.l2scale[b] = nrm > sg2 ? sg2 / nrm : 1.0;
    sc.bf[b][BF_L2SCALE] = (float)sc.l2scale[b];
  }
  if (bd.type == BT_ANNULUS) {  // radial scaling onto the nearer sphere; w = 0 stays 0
    const double nrm = sqrt(ldv(&a[A_WNORM]));
    sc.l2scale[b] = nrm > bd.hi ? bd.hi / nrm : (nrm > 0.0 && nrm < bd.lo ? bd.lo / nrm : 1.0);
    sc.bf[b][BF_L2SCALE] = (float)sc.l2scale[b];
  }
  if (bd.job_w >= 0) {
    JobScal &js = jscal[bd.job_w];
    js.active = 1;
    js.pass = 0;
    js.prefix = 0;
    js.n_above = 0;
    js.c_above = js.s1_above = js.s2_above = 0.0;
    js.tie_needed = 0;
    if (bd.type == BT_L1) {
      js.tau = sc.sigma[b];
      js.theta = 0.0;
      js.mode = js.tau == 0.0 ? JM_NONE : (ldv(&a[A_WNORM]) <= js.tau ? JM_ALL : JM_SELECT);
    } else {
      js.k = sc.kcard[b];
      js.mode = js.k == 0 ? JM_NONE : (js.k >= bd.M ? JM_ALL : JM_SELECT);
    }
  }
  if (bd.job_s >= 0) {
    JobScal &js = jscal[bd.job_s];
    js.active = chk ? 1 : 0;
    js.pass = 0;
    js.prefix = 0;
    js.n_above = 0;
    js.c_above = js.s1_above = js.s2_above = 0.0;
    js.tie_needed = 0;
    if (bd.type == BT_L1) {
      js.tau = sc.sigma[b];
      js.theta = 0.0;
      js.mode = js.tau == 0.0 ? JM_NONE : (ldv(&a[A_S1]) <= js.tau ? JM_ALL : JM_SELECT);
    } else {
      js.k = sc.kcard[b];
      js.mode = js.k == 0 ? JM_NONE : (js.k >= bd.M ? JM_ALL : JM_SELECT);
    }
  }
}

template <typename T, bool ONE, bool BL = false>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 3) k_setpass(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                      InstScal *__restrict__ scal, JobScal *__restrict__ jscal,
                                                      const JobDev *__restrict__ jobs, unsigned long long *ts,
                                                      const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  body_setpass<T, BL>(tiles[blockIdx.x], ONE ? &one.d : insts, scal, jscal, jobs);
}

// --------------------------------------------------------------------------
// Radix selection (l1-ball threshold; top-k).  Keys are the bits of |value|,
// which order like the values.  Pass p histograms one 11-bit digit of the
// entries whose higher digits equal the prefix fixed so far; the last CTA of
// the job picks the bin holding the breakpoint and descends into it.
//   l1:  largest bin d with g(lo_d) >= tau, g(t) = sum_{|w|>t} (|w| - t):
//        the soft threshold theta lies at or above lo_d (Duchi et al.).
//   top-k: largest bin d with count(keys >= lo_d) >= k.
// Bin counts are exact integers; bin sums of |w| (l1) and of w^2 (the
// feasibility measure of the l1 and card sets) are binary64.
// --------------------------------------------------------------------------
// Bin accumulators.  binary32 data: every value in a bin shares one exponent
// E (the first digit holds all exponent bits), so |w| = sig * 2^(E' - 150)
// with an integer significand sig < 2^24 (E' = max(E, 1)); a CTA adds sig
// and sig^2 in 12-bit chunks (2 and 4 of them) with 32-bit shared-memory
// atomics, exact while a work item has at most kMaxChunk rows
// (kMaxChunk * 4095 < 2^32), and folds them into 64-bit global bin sums of
// sig and of sig^2 (the latter as hi * 2^22 + lo).  (64-bit shared-memory
// additions would retry under the contention of the few hot bins.)
// binary64 data: binary64 bin sums.
static_assert((uint64_t)kMaxChunk * 4095u < (1ull << 32), "12-bit chunk sums must fit 32 bits");
template <typename T> struct BinAcc;
template <> struct BinAcc<float> {
  using S = unsigned long long;
  static constexpr size_t kSmem = kBins * 7 * sizeof(uint32_t);  // count, 2 + 4 chunk sums
};
template <> struct BinAcc<double> {
  using S = double;
  static constexpr size_t kSmem = kBins * (sizeof(uint32_t) + 2 * sizeof(S));
};

__device__ __forceinline__ double pow2(int k) {  // 2^k, -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// inclusive suffix sum over the CTA's threads (thread t gets sum_{t' >= t})
__device__ __forceinline__ double cta_suffix(double x, double *wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += v;
  }
  if (lane == 0) wsum[wid] = x;
  __syncthreads();
  double above = 0.0;
  for (int w = wid + 1; w < kThreads / 32; ++w) above += wsum[w];
  __syncthreads();
  return x + above;
}

__device__ __forceinline__ unsigned long long cta_suffix_u64(unsigned long long x, unsigned long long *wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += v;
  }
  if (lane == 0) wsum[wid] = x;
  __syncthreads();
  unsigned long long above = 0;
  for (int w = wid + 1; w < kThreads / 32; ++w) above += wsum[w];
  __syncthreads();
  return x + above;
}

// ---- bin choice by the last CTA of a pass ---------------------------------
// Thread t owns bins [t*kPer, t*kPer + kPer); bins are visited from the top.
//   l1:    largest bin d with g(lo_d) >= tau, g(t) = sum_{|w| >= t} (|w| - t)
//   top-k: largest bin d with count(keys >= lo_d) >= k
// The winner records the entries above the chosen bin (count, sum of |w|,
// sum of w^2) and the new prefix; after the last digit, theta (l1) or the
// k-th key and its tie count (top-k).
constexpr int kPer = kBins / kThreads;

// binary32 keys: integer arithmetic.  A thread's bins share one exponent
// (pass 0: exponent field = thread index; later passes: the prefix's), so
// its bin sums of sig are exact integers in units of 2^e.  Across threads
// pass 0 adds binary64 values (different exponents), later passes integers.
// The l1 test  S_j - cge_j * sig_lo_j >= R  compares an exact integer with
// R = ceil((tau - sums above, binary64) / 2^e).
__device__ __noinline__ void select_choose_int(const JobDev &jd, JobScal &js, const uint32_t *gc,
                                               const unsigned long long *g1, const unsigned long long *g2,
                                               const unsigned long long *g3, int pass, uint32_t pre, int lo,
                                               int nbins, bool need1, bool need2) {
  using U = unsigned long long;
  __shared__ U wsumi[kThreads / 32];
  __shared__ double wsum[kThreads / 32];
  __shared__ int sbest;
  if (threadIdx.x == 0) sbest = -1;
  const bool l1 = jd.kind == JOB_L1;
  U cb[kPer], s1b[kPer], h2b[kPer], l2b[kPer];
  U tc = 0, t1 = 0, th = 0, tl2 = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int bi = threadIdx.x * kPer + j;
    const bool ok = bi < nbins;
    cb[j] = ok ? (U)__ldcg(&gc[bi]) : 0ull;
    s1b[j] = (ok && need1) ? __ldcg(&g1[bi]) : 0ull;
    h2b[j] = (ok && need2) ? __ldcg(&g2[bi]) : 0ull;
    l2b[j] = (ok && need2) ? __ldcg(&g3[bi]) : 0ull;
    tc += cb[j];
    t1 += s1b[j];
    th += h2b[j];
    tl2 += l2b[j];
  }
  // entries strictly above this thread's bins
  U ac = js.n_above + (cta_suffix_u64(tc, wsumi) - tc);
  const int ef = pass == 0 ? (int)threadIdx.x : (int)(pre >> 23);  // exponent field of this thread's bins
  const int e2 = (ef > 0 ? ef : 1) - 150;                          // |w| = sig * 2^e2
  double as1 = js.s1_above, as2 = js.s2_above;  // binary64 sums above (pass 0: incl. higher threads)
  U cs1 = 0, ch2 = 0, cl2 = 0;                  // integer sums above, this pass (later passes: incl. higher threads)
  if (pass == 0) {
    if (need1) {
      const double v = (double)t1 * pow2(e2);
      as1 += cta_suffix(v, wsum) - v;
    }
    if (need2) {
      const double v = ((double)th * 4194304.0 + (double)tl2) * pow2(2 * e2);
      as2 += cta_suffix(v, wsum) - v;
    }
  } else {
    if (need1) cs1 = cta_suffix_u64(t1, wsumi) - t1;
    if (need2) {
      ch2 = cta_suffix_u64(th, wsumi) - th;
      cl2 = cta_suffix_u64(tl2, wsumi) - tl2;
    }
  }
  long long R = 0;
  if (l1) {
    const double r = (js.tau - as1) * pow2(-e2);
    R = r <= -4.0e18 ? -(1ll << 62) : (r >= 4.0e18 ? (1ll << 62) : (long long)ceil(r));
  }
  int best = -1, bj = 0;
  U bc = 0, bs1 = 0, bh2 = 0, bl2 = 0;
  for (int j = kPer - 1; j >= 0; --j) {
    const int bi = threadIdx.x * kPer + j;
    if (bi >= nbins) continue;
    const U cge = ac + cb[j];
    bool ok;
    if (l1) {
      const uint32_t klo = pre | ((uint32_t)bi << lo);
      const uint32_t exl = klo >> 23, manl = klo & 0x7fffffu;
      const U siglo = exl ? (manl | 0x800000u) : manl;
      ok = (long long)(cs1 + s1b[j]) - (long long)(cge * siglo) >= R;
    } else {
      ok = cge >= (U)js.k;
    }
    if (ok) {  // bins below also satisfy; keep the highest
      best = bi;
      bj = j;
      bc = ac;
      bs1 = cs1;
      bh2 = ch2;
      bl2 = cl2;
      break;
    }
    ac = cge;
    cs1 += s1b[j];
    ch2 += h2b[j];
    cl2 += l2b[j];
  }
  __syncthreads();
  {
    const int wb = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && wb >= 0) atomicMax(&sbest, wb);
  }
  __syncthreads();
  if (best >= 0 && best == sbest) {
    const uint32_t np = pre | ((uint32_t)best << lo);
    const double s1a = as1 + (double)bs1 * pow2(e2);
    js.n_above = bc;
    js.c_above = (double)bc;
    js.s1_above = s1a;
    js.s2_above = as2 + ((double)bh2 * 4194304.0 + (double)bl2) * pow2(2 * e2);
    js.prefix = (uint64_t)np;
    if (lo == 0) {  // final digit: the breakpoint key is exact
      if (l1) {
        js.theta = (s1a - js.tau) / (double)bc;
        js.thetaf = (float)js.theta;
      } else {
        js.need = js.k - (int64_t)bc;
        js.cK = (int64_t)cb[bj];
        js.kval = (double)__uint_as_float(np);
        js.tie_needed = (js.need < js.cK && np != 0) ? 1 : 0;
      }
    }
    js.pass = pass + 1;
  }
}

// binary64 keys: binary64 bin sums.
template <typename T>
__device__ __noinline__ void select_choose_f64(const JobDev &jd, JobScal &js, const uint32_t *gc, const double *g1,
                                               const double *g2, int pass, uint64_t pre_, int lo, int nbins,
                                               bool need1, bool need2) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  const K pre = (K)pre_;
  double c[kPer], a1[kPer], a2[kPer];
  double tc = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int bi = threadIdx.x * kPer + j;
    c[j] = a1[j] = a2[j] = 0.0;
    if (bi < nbins) {
      c[j] = (double)__ldcg(&gc[bi]);
      if (need1) a1[j] = __ldcg(&g1[bi]);
      if (need2) a2[j] = __ldcg(&g2[bi]);
    }
    tc += c[j];
    t1 += a1[j];
    t2 += a2[j];
  }
  __shared__ double wsum[kThreads / 32];
  __shared__ unsigned long long wsumi[kThreads / 32];
  // exclusive suffix sums: entries in bins above this thread's range
  const unsigned long long tci = (unsigned long long)tc;
  double ac = js.c_above + (double)(cta_suffix_u64(tci, wsumi) - tci);
  double as1 = js.s1_above, as2 = js.s2_above;
  if (need1) as1 += cta_suffix(t1, wsum) - t1;
  if (need2) as2 += cta_suffix(t2, wsum) - t2;
  int best = -1;
  double bc = 0, b1 = 0, b2 = 0;  // "above" sums for the chosen bin
  for (int j = kPer - 1; j >= 0; --j) {
    const int bi = threadIdx.x * kPer + j;
    if (bi < nbins) {
      const double cge = ac + c[j];
      bool ok;
      if (jd.kind == JOB_L1) {
        const double lov = KT::val(pre | ((K)bi << lo));
        ok = (as1 + a1[j]) - cge * lov >= js.tau;
      } else {
        ok = cge >= (double)js.k;
      }
      if (ok) {  // bins below also satisfy; keep the highest
        best = bi;
        bc = ac;
        b1 = as1;
        b2 = as2;
        break;
      }
    }
    ac += c[j];
    as1 += a1[j];
    as2 += a2[j];
  }
  __shared__ int sbest;
  if (threadIdx.x == 0) sbest = -1;
  __syncthreads();
  {
    const int wb = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && wb >= 0) atomicMax(&sbest, wb);
  }
  __syncthreads();
  if (best >= 0 && best == sbest) {
    const int j = best - threadIdx.x * kPer;
    js.c_above = bc;
    js.n_above = (unsigned long long)bc;
    js.s1_above = b1;
    js.s2_above = b2;
    const K np = pre | ((K)best << lo);
    js.prefix = (uint64_t)np;
    if (lo == 0) {  // final digit: the breakpoint key is exact
      if (jd.kind == JOB_L1) {
        js.theta = (b1 - js.tau) / bc;
        js.thetaf = (float)js.theta;
      } else {
        js.need = js.k - (int64_t)bc;
        js.cK = (int64_t)c[j];
        js.kval = KT::val(np);
        js.tie_needed = (js.need < js.cK && np != 0) ? 1 : 0;
      }
    }
    js.pass = pass + 1;
  }
}

// Top-k from the window candidates (one CTA): the k-th key overall is the
// (k - above)-th largest candidate when above < k <= above + n.  Radix
// passes over the candidates in shared memory, from the highest bit in
// which the window's bounds differ (all candidates share the bits above
// it).  Leaves the job as the last radix pass does.
static_assert((size_t)kWinCap * sizeof(uint32_t) + kBins * sizeof(uint32_t) <= BinAcc<float>::kSmem,
              "binary32 window candidates fit the select kernel's shared memory");
static_assert((size_t)kWinCap * sizeof(uint64_t) + kBins * sizeof(uint32_t) <= BinAcc<double>::kSmem,
              "binary64 window candidates fit the select kernel's shared memory");
template <typename T>
__device__ __noinline__ void select_window_finish(const JobDev &jd, JobScal &js, unsigned char *smem) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  constexpr int kKeyBits = (int)sizeof(K) * 8;
  constexpr int kWarps = kThreads / 32;
  static_assert(kWarps * 32 * kPer == kBins, "thread t owns bins [t kPer, t kPer + kPer)");
  K *ck = (K *)smem;
  uint32_t *h = (uint32_t *)(smem + (size_t)kWinCap * sizeof(K));
  __shared__ uint32_t wt[kWarps];
  __shared__ uint32_t s_above, s_cnt;
  __shared__ int s_bin;
  const int n = (int)js.win_n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const K *cand = (const K *)jd.cand;
  for (int i = threadIdx.x; i < n; i += kThreads) ck[i] = __ldcg(&cand[i]);
  for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0u;
  const K wlo = KT::key((T)js.win_lo), whi = KT::key((T)js.win_hi);
  const K diff = wlo ^ whi;
  int top = 0;  // bits below `top` vary among the candidates
  if (diff) top = kKeyBits - (sizeof(K) == 8 ? __clzll((long long)diff) : __clz((int)diff));
  K pre = wlo;
  uint32_t need = (uint32_t)((unsigned long long)js.k - js.win_above);  // rank among the candidates, 1..n
  uint32_t above_c = 0;      // candidates above the k-th key
  uint32_t cK = (uint32_t)n;  // candidates equal to it
  __syncthreads();
  while (top > 0) {
    const int lo = top > kDigitBits ? top - kDigitBits : 0;
    const int nbins = 1 << (top - lo);
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const K key = ck[i];
      if ((key >> top) == (pre >> top)) atomicAdd(&h[(int)((key >> lo) & (K)(nbins - 1))], 1u);
    }
    __syncthreads();
    // counts of this thread's bins (then cleared for the next pass), warp totals
    uint32_t c[kPer], tc = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      c[j] = h[threadIdx.x * kPer + j];
      h[threadIdx.x * kPer + j] = 0u;
      tc += c[j];
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, tc);
    if (lane == 0) wt[wid] = ws;
    __syncthreads();
    // the warp, then the lane, then the bin holding the need-th largest
    uint32_t aw = 0;
#pragma unroll
    for (int w = kWarps - 1; w > wid; --w) aw += wt[w];
    if (aw < need && need <= aw + ws) {
      uint32_t incl = tc;  // this lane's and the higher lanes' counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += v;
      }
      uint32_t ac = aw + incl - tc;
      if (ac < need && need <= ac + tc) {
        for (int j = kPer - 1; j >= 0; --j) {
          if (ac + c[j] >= need) {
            s_bin = threadIdx.x * kPer + j;
            s_above = ac;
            s_cnt = c[j];
            break;
          }
          ac += c[j];
        }
      }
    }
    __syncthreads();
    need -= s_above;
    above_c += s_above;
    cK = s_cnt;
    pre = (K)((pre >> top) << top) | ((K)s_bin << lo);
    top = lo;
  }
  if (threadIdx.x == 0) {
    const unsigned long long nab = js.win_above + above_c;
    js.n_above = nab;
    js.c_above = (double)nab;
    js.prefix = (uint64_t)pre;
    js.need = js.k - (int64_t)nab;
    js.cK = (int64_t)cK;
    js.kval = KT::val(pre);
    js.tie_needed = (js.need < js.cK && pre != 0) ? 1 : 0;
    js.pass = (KT::kBits + kDigitBits - 1) / kDigitBits;  // past the last radix pass
    js.win_hit = 1;
  }
}

template <typename T>
__device__ __forceinline__ void body_select(const Tile &tl, const InstDev *__restrict__ insts,
                                                        InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                        JobScal *__restrict__ jscal, uint32_t *__restrict__ hcnt,
                                                        double *__restrict__ hs1, double *__restrict__ hs2,
                                                        double *__restrict__ hs3, int64_t hstride, int pass) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  using S = typename BinAcc<T>::S;
  using V = typename Vec16<T>::type;
  constexpr bool kInt = sizeof(T) == 4;
  constexpr int VW = (int)(sizeof(V) / sizeof(T));  // values per vector load
  constexpr int VPT = 4;                            // vector loads per thread and round
  const JobDev jd = jobs[tl.item];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  JobScal &js = jscal[tl.item];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= jd.M, 7u, tl.start + tl.len);
  // Histograms: with hstride > 0, pass p uses buffer p % 3 and the job's
  // CTAs clear, one slice each, the buffer of pass p - 1 (whether or not
  // the job selects in this pass), so every buffer is zero before its next
  // use; with hstride = 0 one buffer, cleared by the last CTA.
  if (hstride) {
    const int64_t zb = (int64_t)((pass + 2) % 3) * hstride + jd.hist_off;
    const int z0 = (int)((int64_t)tl.seq * kBins / jd.ntiles), z1 = (int)((int64_t)(tl.seq + 1) * kBins / jd.ntiles);
    for (int i = z0 + (int)threadIdx.x; i < z1; i += kThreads) {
      hcnt[zb + i] = 0u;
      hs1[zb + i] = 0.0;
      hs2[zb + i] = 0.0;
      hs3[zb + i] = 0.0;
    }
  }
  if (sc.done || !js.active || js.mode != JM_SELECT || js.pass != pass) return;
  extern __shared__ unsigned char smem_raw[];
  if (pass == 0 && jd.kind == JOB_TOPK && !jd.feas && js.win_on) {
    // the k-th key inside this iteration's window: one CTA selects it from
    // the candidates, the radix passes are skipped
    const unsigned long long n = js.win_n, above = js.win_above, kk = (unsigned long long)js.k;
    if (n <= (unsigned long long)kWinCap && above < kk && kk <= above + n) {
      if (tl.seq == 0) select_window_finish<T>(jd, js, smem_raw);
      return;
    }
  }

  uint32_t *cnt = (uint32_t *)smem_raw;
  // binary32: 12-bit chunk sums u[0..1] of sig, u[2..5] of sig^2
  uint32_t *u = cnt + kBins;
  // binary64: sums of |w| and of w^2
  S *s1 = (S *)(smem_raw + kBins * sizeof(uint32_t));
  S *s2 = s1 + kBins;
  const bool need1 = jd.kind == JOB_L1;
  const bool need2 = jd.feas != 0;
  const int hi = KT::kBits - pass * kDigitBits;
  const int lo = hi - kDigitBits > 0 ? hi - kDigitBits : 0;
  const int nbins = 1 << (hi - lo);
  for (int i = threadIdx.x; i < nbins; i += kThreads) {
    cnt[i] = 0;
    if constexpr (kInt) {
      if (need1) u[i] = u[kBins + i] = 0;
      if (need2)
#pragma unroll
        for (int c = 2; c < 6; ++c) u[c * kBins + i] = 0;
    } else {
      if (need1) s1[i] = S(0);
      if (need2) s2[i] = S(0);
    }
  }
  __syncthreads();

  const K mask = (K)(nbins - 1);
  const K pre = (K)js.prefix;
  const bool all = hi >= KT::kBits;
  const T *__restrict__ data = (const T *)(jd.feas ? in.s : in.w) + jd.data_off;
  const int lane = threadIdx.x & 31;
  const int64_t end = tl.start + tl.len;
  // one entry into this CTA's histogram (called by all lanes of a warp)
  auto add = [&](T val, bool valid) {
    int bin = -1;
    K key = 0;
    if (valid) {
      key = KT::key(val);
      if (all || (key >> hi) == (pre >> hi)) bin = (int)((key >> lo) & mask);
    }
    if constexpr (kInt) {
      // exact integer significand and its square in 12-bit chunks
      if (bin >= 0) {
        const uint32_t ex = (uint32_t)key >> 23, man = (uint32_t)key & 0x7fffffu;
        const uint32_t sig = ex ? (man | 0x800000u) : man;
        atomicAdd(&cnt[bin], 1u);
        if (need1) {
          atomicAdd(&u[bin], sig & 0xfffu);
          atomicAdd(&u[kBins + bin], sig >> 12);
        }
        if (need2) {
          const uint64_t sq = (uint64_t)sig * sig;
#pragma unroll
          for (int c = 0; c < 4; ++c) atomicAdd(&u[(2 + c) * kBins + bin], (uint32_t)(sq >> (12 * c)) & 0xfffu);
        }
      }
    } else {
      unsigned pending = __ballot_sync(0xffffffffu, bin >= 0);
      const double a = bin >= 0 ? fabs((double)val) : 0.0;
      while (pending) {
        const int leader = __ffs(pending) - 1;
        const int lb = __shfl_sync(0xffffffffu, bin, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, bin == lb);
        const bool mine = bin == lb;
        double v1 = 0.0, v2 = 0.0;
        if (need1) v1 = warp_sum(mine ? a : 0.0);
        if (need2) v2 = warp_sum(mine ? a * a : 0.0);
        if (lane == leader) {
          atomicAdd(&cnt[lb], (uint32_t)__popc(grp));
          if (need1) atomicAdd((double *)&s1[lb], v1);
          if (need2) atomicAdd((double *)&s2[lb], v2);
        }
        pending &= ~grp;
      }
    }
  };
  if (((uintptr_t)(data + tl.start) & (sizeof(V) - 1)) == 0) {
    // 16-byte loads (a vector that reaches past the work item is read one
    // value at a time)
    for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * VW * VPT) {
      V v[VPT];
#pragma unroll
      for (int e = 0; e < VPT; ++e) {
        const int64_t i0 = base + (int64_t)(threadIdx.x + e * kThreads) * VW;
        if (i0 + VW <= end) {
          v[e] = *(const V *)(data + i0);
        } else {
#pragma unroll
          for (int c = 0; c < VW; ++c) vset(v[e], c, i0 + c < end ? data[i0 + c] : T(0));
        }
      }
#pragma unroll
      for (int e = 0; e < VPT; ++e) {
        const int64_t i0 = base + (int64_t)(threadIdx.x + e * kThreads) * VW;
#pragma unroll
        for (int c = 0; c < VW; ++c) add(vat(v[e], c), i0 + c < end);
      }
    }
  } else {
    constexpr int PT = 4;
    for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * PT) {
      T val[PT];
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
        val[e] = row < end ? data[row] : T(0);
      }
#pragma unroll
      for (int e = 0; e < PT; ++e) add(val[e], base + threadIdx.x + (int64_t)e * kThreads < end);
    }
  }
  __syncthreads();
  const int64_t hb = (hstride ? (int64_t)(pass % 3) * hstride : 0) + jd.hist_off;
  uint32_t *gc = hcnt + hb;
  S *g1 = (S *)(hs1 + hb);
  S *g2 = (S *)(hs2 + hb);
  S *g3 = (S *)(hs3 + hb);
  for (int i = threadIdx.x; i < nbins; i += kThreads) {
    const uint32_t c = cnt[i];
    if (c) {
      atomicAdd(&gc[i], c);
      if constexpr (kInt) {
        if (need1) atomicAdd(&g1[i], (S)u[i] + ((S)u[kBins + i] << 12));
        if (need2) {
          // sum of sig^2 = lo24 + Q2 2^24 + Q3 2^36 = hi * 2^22 + (lo24 mod 2^22)
          const S lo24 = (S)u[2 * kBins + i] + ((S)u[3 * kBins + i] << 12);
          atomicAdd(&g2[i], (lo24 >> 22) + ((S)u[4 * kBins + i] << 2) + ((S)u[5 * kBins + i] << 14));
          atomicAdd(&g3[i], lo24 & 0x3fffffull);
        }
      } else {
        if (need1) atomicAdd(&g1[i], s1[i]);
        if (need2) atomicAdd(&g2[i], s2[i]);
      }
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = arrive_last(&js.counter, (uint32_t)jd.ntiles);
  __syncthreads();
  if (!last) return;

  if constexpr (kInt) {
    select_choose_int(jd, js, gc, (const S *)g1, (const S *)g2, (const S *)g3, pass, pre, lo, nbins, need1, need2);
  } else {
    select_choose_f64<T>(jd, js, gc, g1, g2, pass, pre, lo, nbins, need1, need2);
  }
  if (hstride) return;
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += kThreads) {
    gc[i] = 0;
    if (need1) g1[i] = S(0);
    if (need2) {
      g2[i] = S(0);
      if (kInt) g3[i] = S(0);
    }
  }
}

template <typename T, bool ONE>
__global__ void __launch_bounds__(kThreads, 3) k_select(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                        InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                        JobScal *__restrict__ jscal, uint32_t *__restrict__ hcnt,
                                                        double *__restrict__ hs1, double *__restrict__ hs2,
                                                        double *__restrict__ hs3, int64_t hstride, int pass,
                                                        unsigned long long *ts, const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  body_select<T>(tiles[blockIdx.x], ONE ? &one.d : insts, scal, jobs, jscal, hcnt, hs1, hs2, hs3, hstride, pass);
}

// Tie counts per final-pass work item for card sets whose k-th value is tied.
template <typename T>
__device__ __forceinline__ void body_ties(const Tile &tl, const InstDev *__restrict__ insts,
                                                   InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                   JobScal *__restrict__ jscal, uint32_t *__restrict__ ties) {
  SIP_STEP_CONSTANTS;
  using KT = KeyOf<T>;
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  const BlockDev &bd = in.blk[tl.item];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= bd.M, 8u, tl.start + tl.len);
  if (sc.done || bd.type != BT_CARD) return;
  const JobScal &js = jscal[bd.job_w];
  if (js.mode != JM_SELECT || !js.tie_needed) return;
  const typename KT::K K = (typename KT::K)js.prefix;
  const T *__restrict__ w = (const T *)in.w + bd.woff;
  const int64_t end = tl.start + tl.len;
  int n = 0;
  for (int64_t base = tl.start; base < end; base += SUB) {
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
      if (row < end && KT::key(w[row]) == K) ++n;
    }
  }
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  if (n) atomicAdd(&tot, n);
  __syncthreads();
  if (threadIdx.x == 0) ties[jobs[bd.job_w].tie_off + tl.seq] = (uint32_t)tot;
}

template <typename T, bool ONE>
__global__ void __launch_bounds__(kThreads, 4) k_ties(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                   InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                   JobScal *__restrict__ jscal, uint32_t *__restrict__ ties, unsigned long long *ts,
                                                   const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  body_ties<T>(tiles[blockIdx.x], ONE ? &one.d : insts, scal, jobs, jscal, ties);
}

// --------------------------------------------------------------------------
// Final pass: l1 / l2 / card prox from the stored w and the dual update
// v = v + rho (y - xbar) = rho (y - w), since w = xbar - v / rho.
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void body_final(const Tile &tl, const InstDev *__restrict__ insts,
                                                    InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                    const JobScal *__restrict__ jscal,
                                                    const uint32_t *__restrict__ ties) {
  SIP_STEP_CONSTANTS;
  using KT = KeyOf<T>;
  using K = typename KT::K;
  using A = typename AccOf<T>::type;
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  const int b = tl.item;
  const BlockDev &bd = in.blk[b];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= bd.M, 9u, tl.start + tl.len);
  // binary32: the first round's w is requested before the instance's and
  // the job's state arrive (used by the 16-byte path, discarded otherwise)
  constexpr int FU = 2;
  float4 W0[FU];
  bool w0_ok = false;
  if constexpr (sizeof(T) == 4) {
    const float *w0 = (const float *)in.w + bd.woff;
    const int64_t e0 = tl.start + tl.len;
    w0_ok = ((uintptr_t)(w0 + tl.start) & 15) == 0;
    if (w0_ok) {
#pragma unroll
      for (int h = 0; h < FU; ++h) {
        const int64_t r0 = tl.start + ((int64_t)h * kThreads + threadIdx.x) * 4;
        W0[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + 4 <= e0) {
          W0[h] = ld4(w0, r0);
        } else {
          for (int c = 0; c < 4; ++c)
            if (r0 + c < e0) vset(W0[h], c, w0[r0 + c]);
        }
      }
    }
  }
  if (sc.done) return;
  const int k = sc.k;
  const bool ad = adapt_iter(in, k);
  const bool ad_dots = ad && sc.have_k0;
  const T rho = SV<T>::blk(sc, b, BF_RHO);
  const T *__restrict__ w = (const T *)in.w + bd.woff;
  T *__restrict__ y = (T *)in.y + bd.yoff;
  T *__restrict__ v = (T *)in.v + bd.yoff;
  T *__restrict__ k0y = (T *)in.k0y + bd.yoff;
  T *__restrict__ k0v = (T *)in.k0v + bd.yoff;
  int mode = JM_ALL;
  T theta = T(0);
  K K0 = 0;
  bool tie = false;
  int64_t need = 0, before = 0;
  if (bd.type != BT_L2 && bd.type != BT_ANNULUS) {
    const JobScal &js = jscal[bd.job_w];
    mode = js.mode;
    theta = SV<T>::theta(js);
    K0 = (K)js.prefix;
    tie = bd.type == BT_CARD && mode == JM_SELECT && js.tie_needed;
    need = js.need;
    if (tie) {  // ties in earlier work items of this block
      const uint32_t *tc = ties + jobs[bd.job_w].tie_off;
      for (int i = threadIdx.x; i < tl.seq; i += kThreads) before += tc[i];
      __shared__ unsigned long long sb;
      if (threadIdx.x == 0) sb = 0;
      __syncthreads();
      if (before) atomicAdd(&sb, (unsigned long long)before);
      __syncthreads();
      before = (int64_t)sb;
    }
  }
  const T scale = SV<T>::blk(sc, b, BF_L2SCALE);
  // l2 data fit: observed values d (NaN: unobserved), y = d + scale (w - d)
  const T *__restrict__ cen = (bd.type == BT_L2 && bd.bv_lo >= 0) ? (const T *)in.bvec + bd.bv_lo : nullptr;
  const T th = theta;
  const int type = bd.type;
  A acc[3] = {A(0), A(0), A(0)};
  __shared__ int wcount[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t end = tl.start + tl.len;
  // prox of one entry (no tie rank)
  auto prox = [&](T wv) -> T {
    if (type == BT_L2 || type == BT_ANNULUS) return wv * scale;
    if (mode == JM_ALL) return wv;
    if (mode == JM_NONE) return T(0);
    if (type == BT_L1) {
      const T a = fabs(wv) - th;
      return a > T(0) ? copysign(a, wv) : T(0);
    }
    return KT::key(wv) >= K0 ? wv : T(0);  // card, no tie at the k-th key
  };
  bool vec = false;
  if constexpr (sizeof(T) == 4) {
    uintptr_t al = (uintptr_t)(w + tl.start) | (uintptr_t)(y + tl.start) | (uintptr_t)(v + tl.start);
    if (ad) al |= (uintptr_t)(k0y + tl.start) | (uintptr_t)(k0v + tl.start);
    vec = !tie && !cen && (al & 15) == 0;
  }
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      // 16-byte accesses, 4 consecutive rows per thread, two groups of 4
      // per round (their loads requested together)
      for (int64_t base = tl.start; base < end; base += (int64_t)kThreads * 4 * FU) {
        auto ld = [&](const float *p, int64_t r0) {
          if (r0 + 4 <= end) return ld4(p, r0);
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int c = 0; c < 4; ++c)
            if (r0 + c < end) vset(t, c, p[r0 + c]);
          return t;
        };
        auto st = [&](float *p, int64_t r0, const float4 &t) {
          if (r0 + 4 <= end) {
            st4(p, r0, t);
          } else {
            for (int c = 0; c < 4; ++c)
              if (r0 + c < end) p[r0 + c] = vat(t, c);
          }
        };
        float4 W[FU], KY[FU], KV[FU];
#pragma unroll
        for (int h = 0; h < FU; ++h) {
          const int64_t r0 = base + ((int64_t)h * kThreads + threadIdx.x) * 4;
          W[h] = KY[h] = KV[h] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (r0 < end) {
            W[h] = (base == tl.start && w0_ok) ? W0[h] : ld(w, r0);
            if (ad_dots) {
              KY[h] = ld(k0y, r0);
              KV[h] = ld(k0v, r0);
            }
          }
        }
#pragma unroll
        for (int h = 0; h < FU; ++h) {
          const int64_t r0 = base + ((int64_t)h * kThreads + threadIdx.x) * 4;
          if (r0 >= end) continue;
          float4 YN, VN;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float wc = vat(W[h], c);
            const float yn = prox(wc), vn = rho * (yn - wc);
            vset(YN, c, yn);
            vset(VN, c, vn);
            if (ad_dots && r0 + c < end) {
              const A dg = (A)vat(KY[h], c) - (A)yn;
              const A dv = (A)vn - (A)vat(KV[h], c);
              acc[0] += dg * dv;
              acc[1] += dg * dg;
              acc[2] += dv * dv;
            }
          }
          if (in.bf16) {
            YN = rbf4(YN);
            VN = rbf4(VN);
          }
          st(y, r0, YN);
          st(v, r0, VN);
          if (ad) {
            st(k0y, r0, YN);
            st(k0v, r0, VN);
          }
        }
      }
    }
  } else {
    for (int64_t base = tl.start; base < end; base += SUB) {
      T wv[PT], ky[PT], kv[PT];
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
        if (row < end) {
          wv[e] = w[row];
          if (ad_dots) {
            ky[e] = k0y[row];
            kv[e] = k0v[row];
          }
        } else {
          wv[e] = T(0);
        }
      }
#pragma unroll
      for (int e = 0; e < PT; ++e) {
        const int64_t row = base + threadIdx.x + (int64_t)e * kThreads;
        const bool valid = row < end;
        T yn;
        if (cen) {
          const T c = valid ? cen[row] : T(0);
          yn = isnan(c) ? wv[e] : c + (wv[e] - c) * scale;
        } else if (type == BT_L2 || type == BT_ANNULUS) {
          yn = wv[e] * scale;
        } else if (mode == JM_ALL) {
          yn = wv[e];
        } else if (mode == JM_NONE) {
          yn = T(0);
        } else if (type == BT_L1) {
          const T a = fabs(wv[e]) - th;
          yn = a > T(0) ? copysign(a, wv[e]) : T(0);
        } else {
          // card: keep keys above the k-th key; at the k-th key keep all ties
          // unless the tie rule must choose (ranked below)
          const K key = KT::key(wv[e]);
          yn = (key > K0 || (key == K0 && !tie)) ? wv[e] : T(0);
        }
        if (tie) {
          // rank among tied entries in row order: rows are ordered by
          // (step, e, thread), so scan this round's flags over the CTA
          const bool f = valid && KT::key(wv[e]) == K0;
          const unsigned bal = __ballot_sync(0xffffffffu, f);
          if (lane == 0) wcount[wid] = __popc(bal);
          __syncthreads();
          int pre = 0, total = 0;
          for (int i = 0; i < kThreads / 32; ++i) {
            if (i < wid) pre += wcount[i];
            total += wcount[i];
          }
          const int64_t rank = before + pre + __popc(bal & ((1u << lane) - 1u));
          if (f) yn = rank < need ? wv[e] : T(0);
          before += total;
          __syncthreads();
        }
        if (valid) {
          const T vn = rho * (yn - wv[e]);
          const T yst = in.bf16 ? rbf(yn) : yn, vst = in.bf16 ? rbf(vn) : vn;
          y[row] = yst;
          v[row] = vst;
          if (ad) {
            if (ad_dots) {
              const A dg = (A)ky[e] - (A)yn;
              const A dv = (A)vn - (A)kv[e];
              acc[0] += dg * dv;
              acc[1] += dg * dg;
              acc[2] += dv * dv;
            }
            k0y[row] = yst;
            k0v[row] = vst;
          }
        }
      }
    }
  }
  if (ad_dots) {
    block_sum<3>(acc);
    if (threadIdx.x == 0) {
      atomicAdd(&sc.acc[b][A_GV], (double)acc[0]);
      atomicAdd(&sc.acc[b][A_GG], (double)acc[1]);
      atomicAdd(&sc.acc[b][A_VV], (double)acc[2]);
    }
  }
}

template <typename T, bool ONE>
__global__ void __launch_bounds__(kThreads, 4) k_final(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                    InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                    const JobScal *__restrict__ jscal,
                                                    const uint32_t *__restrict__ ties, unsigned long long *ts,
                                                    const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  body_final<T>(tiles[blockIdx.x], ONE ? &one.d : insts, scal, jobs, jscal, ties);
}

// --------------------------------------------------------------------------
// Per-line sets: the simple set's projection of every line of A x along z, x
// or y on its own (the paper's per-column / per-row / per-fiber sets).  One
// CTA projects one line at a time: l2 and annulus from the line's norm;
// card and l1 from the line sorted by (|value| decreasing, position
// increasing), a bitonic sort in shared memory (lines of at most
// kLineMax entries).  Then the dual update v = rho (y - w) and the adapt
// sums as in the final pass; on check iterations the same projection of s
// gives the feasibility distance.
// --------------------------------------------------------------------------
constexpr int kLineMax = SIP_MAX_LINE;
constexpr int kLineSmallK = 8;  // per-line top-k by per-thread lists up to this k
template <typename T>
constexpr size_t line_smem() {
  return (size_t)kLineMax * (sizeof(typename KeyOf<T>::K) + sizeof(uint32_t) + 1);
}

// (key, position) pairs in decreasing key order, equal keys by position.
template <typename K>
__device__ void cta_sort_desc(K *key, uint32_t *pos, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kThreads) {
        const int q = i ^ j;
        if (q > i) {
          const K ki = key[i], kq = key[q];
          const uint32_t pi = pos[i], pq = pos[q];
          const bool i_first = ki > kq || (ki == kq && pi < pq);
          if (((i & k) == 0) != i_first) {
            key[i] = kq;
            key[q] = ki;
            pos[i] = pq;
            pos[q] = pi;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Block-wide sum in binary64, fixed order.
__device__ __forceinline__ double cta_sum_f64(double x, double *red) {
  double a[1] = {x};
  block_sum<1>(a);
  if (threadIdx.x == 0) red[0] = a[0];
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// Projection of one line of src (len entries, stride apart from base).
// out == true: y = P(w), v = rho (y - w), adapt sums into ac; otherwise
// (s on a check iteration) the squared distance and squared norm into
// *d2, *s2 (thread 0).
template <typename T>
__device__ void line_project(const BlockDev &bd, const T *__restrict__ src, int64_t base, double sigma, int64_t kk,
                             T rho, bool out, bool ad, bool ad_dots, T *__restrict__ y, T *__restrict__ v,
                             T *__restrict__ k0y, T *__restrict__ k0v, typename AccOf<T>::type (&ac)[3],
                             double *d2, double *s2, unsigned char *smem) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  using A = typename AccOf<T>::type;
  __shared__ double red[1];
  __shared__ double s_theta;
  __shared__ int s_best;
  const int64_t L = bd.line_len, S = bd.line_stride;
  const int lt = bd.line_type;
  auto at = [&](int64_t e) { return base + e * S; };
  // mode: 0 scale, 1 keep the flagged entries, 2 soft threshold
  int mode = 0;
  double scale = 1.0;
  double theta = 0.0;
  double ss = 0.0, sa = 0.0;
  // ||line||^2: for the l2 / annulus scale and the feasibility pass;
  // ||line||_1: for the l1 ball
  const bool need_ss = lt == BT_L2 || lt == BT_ANNULUS || !out;
  if (need_ss || lt == BT_L1) {
    for (int64_t e = threadIdx.x; e < L; e += kThreads) {
      const double x = (double)src[at(e)];
      ss += x * x;
      sa += fabs(x);
    }
  }
  if (need_ss) ss = cta_sum_f64(ss, red);
  if (lt == BT_L2 || lt == BT_ANNULUS) {
    const double nrm = sqrt(ss);
    const double hi = lt == BT_L2 ? sigma : bd.hi, lo = lt == BT_L2 ? 0.0 : bd.lo;
    scale = nrm > hi ? hi / nrm : (nrm > 0.0 && nrm < lo ? lo / nrm : 1.0);
  } else if (lt == BT_L1) {
    sa = cta_sum_f64(sa, red);
    if (sigma == 0.0) {
      scale = 0.0;
    } else if (sa > sigma) {
      // theta from the sorted magnitudes u_1 >= u_2 >= ...: the largest j
      // with u_j > (c_j - sigma) / j, c_j the running sum (Duchi et al.)
      K *key = (K *)smem;
      uint32_t *pos = (uint32_t *)(smem + (size_t)kLineMax * sizeof(K));
      int n2 = 1;
      while (n2 < L) n2 <<= 1;
      for (int i = threadIdx.x; i < n2; i += kThreads) {
        key[i] = i < L ? KT::key(src[at(i)]) : K(0);
        pos[i] = (uint32_t)i;
      }
      __syncthreads();
      cta_sort_desc(key, pos, n2);
      // each thread sums a run of sorted entries; exclusive scan of the runs
      const int per = (int)((L + kThreads - 1) / kThreads);
      const int i0 = threadIdx.x * per, i1 = (int)(i0 + per < L ? i0 + per : L);
      double run = 0.0;
      for (int i = i0; i < i1; ++i) run += KT::val(key[i]);
      __shared__ double wrun[kThreads];
      wrun[threadIdx.x] = run;
      if (threadIdx.x == 0) s_best = -1;
      __syncthreads();
      double c = 0.0;
      for (int t = 0; t < (int)threadIdx.x; ++t) c += wrun[t];
      int best = -1;
      double cbest = 0.0;
      for (int i = i0; i < i1; ++i) {
        const double u = KT::val(key[i]);
        c += u;
        if (u > (c - sigma) / (double)(i + 1)) {
          best = i;
          cbest = c;
        }
      }
      const int wb = __reduce_max_sync(0xffffffffu, best);
      if ((threadIdx.x & 31) == 0 && wb >= 0) atomicMax(&s_best, wb);
      __syncthreads();
      if (best >= 0 && best == s_best) s_theta = (cbest - sigma) / (double)(best + 1);
      __syncthreads();
      theta = s_theta;
      mode = 2;
    }
  } else {  // card
    if (kk <= 0) {
      scale = 0.0;
    } else if (kk < L) {
      mode = 1;
    }
  }
  // card: the k-th key K by radix passes over the line (11-bit digits, a
  // shared-memory histogram, the bin picked through warp totals); entries
  // above K stay, and of the cK entries equal to K the first `need` in line
  // order.  Thread t then walks positions [t c, (t + 1) c) in order, its
  // tie rank starting at the tied entries of the threads before it.
  K kkey = 0;
  uint32_t need = 0, tie0 = 0;
  bool all_ties = true;
  const int per = (int)((L + kThreads - 1) / kThreads);
  const int e0 = (int)threadIdx.x * per, e1 = (int)(e0 + per < L ? e0 + per : L);
  // small k (the paper's "at most a few nonzeros per row / column"): the
  // line's k largest entries in the order (|w| descending, position
  // ascending) -- the same set as the radix selection with its tie rule --
  // from each thread's own top k over its positions, then k rounds of a
  // CTA-wide maximum; the output keeps exactly the selected positions
  __shared__ uint32_t s_sel[kLineSmallK];
  if (mode == 1 && kk <= kLineSmallK) {
    const int kq = (int)kk;
    K tk[kLineSmallK];
    uint32_t tp[kLineSmallK];
#pragma unroll
    for (int j = 0; j < kLineSmallK; ++j) {
      tk[j] = 0;
      tp[j] = 0xffffffffu;
    }
    // positions ascend within a thread: an entry enters only if its key is
    // strictly larger than the current k-th
    for (int e = e0; e < e1; ++e) {
      const K key = KT::key(src[at(e)]);
      if (tp[kq - 1] != 0xffffffffu && key <= tk[kq - 1]) continue;
      K ck = key;
      uint32_t cp = (uint32_t)e;
#pragma unroll
      for (int j = 0; j < kLineSmallK; ++j) {
        if (j < kq && (tp[j] == 0xffffffffu || ck > tk[j])) {
          const K t1 = tk[j];
          const uint32_t t2 = tp[j];
          tk[j] = ck;
          tp[j] = cp;
          ck = t1;
          cp = t2;
        }
      }
    }
    constexpr int kWarps = kThreads / 32;
    __shared__ K wk[kWarps];
    __shared__ uint32_t wp[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int head = 0;
    for (int round = 0; round < kq; ++round) {
      // this thread's next candidate; exhausted threads offer nothing
      K bk = 0;
      uint32_t bp = 0xffffffffu;
#pragma unroll
      for (int j = 0; j < kLineSmallK; ++j)
        if (j == head) {
          bk = tk[j];
          bp = tp[j];
        }
      if (head >= kq) bp = 0xffffffffu;
      K mk = bk;
      uint32_t mp = bp;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const K ok2 = __shfl_xor_sync(0xffffffffu, mk, o);
        const uint32_t op = __shfl_xor_sync(0xffffffffu, mp, o);
        const bool better = op != 0xffffffffu && (mp == 0xffffffffu || ok2 > mk || (ok2 == mk && op < mp));
        if (better) {
          mk = ok2;
          mp = op;
        }
      }
      if (lane == 0) {
        wk[wid] = mk;
        wp[wid] = mp;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        K gk = wk[0];
        uint32_t gp = wp[0];
        for (int w2 = 1; w2 < kWarps; ++w2)
          if (wp[w2] != 0xffffffffu && (gp == 0xffffffffu || wk[w2] > gk || (wk[w2] == gk && wp[w2] < gp))) {
            gk = wk[w2];
            gp = wp[w2];
          }
        s_sel[round] = gp;
      }
      __syncthreads();
      if (bp != 0xffffffffu && bp == s_sel[round]) ++head;  // positions are unique
    }
    mode = 3;
  }
  if (mode == 1) {
    constexpr int kWarps = kThreads / 32;
    uint32_t *h = (uint32_t *)smem;
    __shared__ uint32_t wt[kWarps];
    __shared__ uint32_t s_above, s_cnt;
    __shared__ int s_bin;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    need = (uint32_t)kk;
    K pre = 0;
    uint32_t cK = 0;
    for (int hi = KT::kBits; hi > 0;) {
      const int lo = hi > kDigitBits ? hi - kDigitBits : 0;
      const int nbins = 1 << (hi - lo);
      for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0u;
      __syncthreads();
      for (int64_t e = threadIdx.x; e < L; e += kThreads) {
        const K key = KT::key(src[at(e)]);
        if (hi == KT::kBits || (key >> hi) == (pre >> hi)) atomicAdd(&h[(int)((key >> lo) & (K)(nbins - 1))], 1u);
      }
      __syncthreads();
      uint32_t c[kPer], tc = 0;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        c[j] = h[threadIdx.x * kPer + j];
        tc += c[j];
      }
      const uint32_t ws = __reduce_add_sync(0xffffffffu, tc);
      if (lane == 0) wt[wid] = ws;
      __syncthreads();
      uint32_t aw = 0;
#pragma unroll
      for (int w2 = kWarps - 1; w2 > wid; --w2) aw += wt[w2];
      if (aw < need && need <= aw + ws) {
        uint32_t incl = tc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v2 = __shfl_down_sync(0xffffffffu, incl, o);
          if (lane + o < 32) incl += v2;
        }
        uint32_t ac = aw + incl - tc;
        if (ac < need && need <= ac + tc) {
          for (int j = kPer - 1; j >= 0; --j) {
            if (ac + c[j] >= need) {
              s_bin = threadIdx.x * kPer + j;
              s_above = ac;
              s_cnt = c[j];
              break;
            }
            ac += c[j];
          }
        }
      }
      __syncthreads();
      need -= s_above;
      cK = s_cnt;
      pre = (K)(pre | ((K)s_bin << lo));
      hi = lo;
      __syncthreads();
    }
    kkey = pre;
    all_ties = need >= cK;
    if (!all_ties) {
      // tied entries before this thread's positions (in line order)
      uint32_t mine = 0;
      for (int e = e0; e < e1; ++e) mine += KT::key(src[at(e)]) == kkey ? 1u : 0u;
      uint32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v2 = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v2;
      }
      if (lane == 31) wt[wid] = incl;
      __syncthreads();
      uint32_t before = 0;
      for (int w2 = 0; w2 < wid; ++w2) before += wt[w2];
      tie0 = before + incl - mine;
      __syncthreads();
    }
  }
  const T sc_t = (T)scale, th = (T)theta;
  double dd = 0.0;
  uint32_t tie = tie0;
  for (int64_t e = (mode == 1 ? e0 : threadIdx.x); e < (mode == 1 ? e1 : L); e += (mode == 1 ? 1 : kThreads)) {
    // (mode 3 walks the line like the point-wise modes)
    const int64_t r = at(e);
    const T wv = src[r];
    T yn;
    if (mode == 1) {
      const K key = KT::key(wv);
      bool keep = key > kkey;
      if (key == kkey) keep = all_ties || tie++ < need;
      yn = keep ? wv : T(0);
    } else if (mode == 3) {
      bool keep = false;
      for (int j = 0; j < (int)kk; ++j) keep = keep || s_sel[j] == (uint32_t)e;
      yn = keep ? wv : T(0);
    } else if (mode == 2) {
      const T a = fabs(wv) - th;
      yn = a > T(0) ? copysign(a, wv) : T(0);
    } else {
      yn = wv * sc_t;
    }
    if (out) {
      const T vn = rho * (yn - wv);
      if (ad_dots) {
        const A dg = (A)k0y[r] - (A)yn;
        const A dv = (A)vn - (A)k0v[r];
        ac[0] += dg * dv;
        ac[1] += dg * dg;
        ac[2] += dv * dv;
      }
      y[r] = yn;
      v[r] = vn;
      if (ad) {
        k0y[r] = yn;
        k0v[r] = vn;
      }
    } else {
      const double d = (double)wv - (double)yn;
      dd += d * d;
    }
  }
  if (!out) {
    dd = cta_sum_f64(dd, red);
    if (threadIdx.x == 0) {
      *d2 += dd;
      *s2 += ss;
    }
  }
  __syncthreads();  // shared arrays are reused by the next line
}

template <typename T>
__device__ __forceinline__ void body_lines(const Tile &tl, const InstDev *__restrict__ insts,
                                           InstScal *__restrict__ scal, unsigned char *smem) {
  using A = typename AccOf<T>::type;
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  const int b = tl.item;
  const BlockDev &bd = in.blk[b];
  SIP_GUARD_TILE(in.err, tl.start >= 0 && tl.start + tl.len <= bd.nlines, 10u, tl.start + tl.len);
  const int k = sc.k;
  const bool ad = adapt_iter(in, k);
  const bool ad_dots = ad && sc.have_k0;
  const bool chk = check_iter(in, k);
  const T rho = SV<T>::blk(sc, b, BF_RHO);
  const double sigma = sc.sigma[b];
  const int64_t kk = sc.kcard[b];
  const T *__restrict__ w = (const T *)in.w + bd.woff;
  const T *__restrict__ s = (const T *)in.s + bd.soff;
  T *__restrict__ y = (T *)in.y + bd.yoff;
  T *__restrict__ v = (T *)in.v + bd.yoff;
  T *__restrict__ k0y = (T *)in.k0y + bd.yoff;
  T *__restrict__ k0v = (T *)in.k0v + bd.yoff;
  A ac[3] = {A(0), A(0), A(0)};
  double d2 = 0.0, s2 = 0.0;
  for (int64_t j = tl.start; j < tl.start + tl.len; ++j) {
    const int64_t base = (j % bd.line_a) + (j / bd.line_a) * bd.line_b;
    line_project<T>(bd, w, base, sigma, kk, rho, true, ad, ad_dots, y, v, k0y, k0v, ac, &d2, &s2, smem);
    if (chk) line_project<T>(bd, s, base, sigma, kk, rho, false, false, false, y, v, k0y, k0v, ac, &d2, &s2, smem);
  }
  if (ad_dots) {
    block_sum<3>(ac);
    if (threadIdx.x == 0) {
      atomicAdd(&sc.acc[b][A_GV], (double)ac[0]);
      atomicAdd(&sc.acc[b][A_GG], (double)ac[1]);
      atomicAdd(&sc.acc[b][A_VV], (double)ac[2]);
    }
  }
  if (chk && threadIdx.x == 0) atomicAdd(&sc.acc[b][A_FEAS_D2], d2);  // ||s||^2: the set pass
}

template <typename T, bool ONE>
__global__ void __launch_bounds__(kThreads, 3) k_lines(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                    InstScal *__restrict__ scal, unsigned long long *ts,
                                                    const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  extern __shared__ unsigned char smem_raw[];
  body_lines<T>(tiles[blockIdx.x], ONE ? &one.d : insts, scal, smem_raw);
}

// --------------------------------------------------------------------------
// Per-instance tail: stopping quantities, Algorithm adapt-rho-gamma, C.
// --------------------------------------------------------------------------
__device__ void set_coefficients(const InstDev &in, InstScal &sc) {
  double c0 = in.alg1 ? 0.0 : 1.0, cz = 0.0, cx = 0.0, cy = 0.0;
  for (int b = 0; b < in.nb; ++b) {
    const double r = sc.rho[b];
    sc.irho[b] = __drcp_rn(r);  // = 1 / r correctly rounded, as the division
    sc.inv1p[b] = __drcp_rn(1.0 + r);
    switch (in.blk[b].op) {
      case SIP_OP_I: c0 += r; break;
      case SIP_OP_DZ: cz += r; break;
      case SIP_OP_DX: cx += r; break;
      case SIP_OP_DY: cy += r; break;
      case SIP_OP_BLUR: break;  // rho_F F^T F: the blur term of the CG launches
      default: cz += r; cx += r; if (in.ndim == 3) cy += r; break;
    }
  }
  sc.c0 = c0;
  sc.cz = cz * in.ihz * in.ihz;
  sc.cx = cx * in.ihx * in.ihx;
  sc.cy = cy * in.ihy * in.ihy;
  store_coef_f32(sc);
  for (int b = 0; b < in.nb; ++b) store_block_f32(sc, b);
}

__device__ __forceinline__ double corr(double ab, double aa, double bb) {
  const double d = aa * bb;
  return d > 0.0 ? ab / sqrt(d) : 0.0;
}
__device__ __forceinline__ double spectral(double ab, double aa, double bb) {
  const double mg = ab / aa, sd = bb / ab;
  return 2.0 * mg > sd ? mg : sd - 0.5 * mg;
}

constexpr int kTailWarps = 8;

__device__ __forceinline__ void body_tail(int i, const InstDev *__restrict__ insts, InstScal *__restrict__ scal,
                                          JobScal *__restrict__ jscal, int cg_launch) {
  const InstDev &in = insts[i];
  InstScal &sc = scal[i];
  if (sc.done) return;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = in.nb, p = in.p;
  const int k = sc.k;
  const bool chk = check_iter(in, k);
  const bool ad = adapt_iter(in, k);
  const bool have_k0 = sc.have_k0 != 0;
  __shared__ double s_rho[kMaxBlocks], s_gam[kMaxBlocks], s_feas[kMaxBlocks];

  // ---- phase 1: per block, warp b % kTailWarps (binary64 chains of
  // different blocks run on different SM sub-partitions).  Within the warp
  // the two correlation tests of Algorithm adapt-rho-gamma and the
  // feasibility run on lanes 0, 1 and 2 at once (binary64 divisions and
  // square roots are long on this GPU), lane 0 combines them.
  for (int b = wid; b < nb; b += kTailWarps) {
    const BlockDev &bd = in.blk[b];
    const double *a = sc.acc[b];
    int ok = 0;
    double hat = 0.0, fe = 0.0;
    if (ad && have_k0 && lane < 2) {
      // lane 0: dh with dvh (alpha); lane 1: dg with dv (beta)
      const double ab = lane == 0 ? a[A_HV] : a[A_GV];
      const double aa = lane == 0 ? a[A_HH] : a[A_GG];
      const double bb = lane == 0 ? a[A_VHVH] : a[A_VV];
      ok = corr(ab, aa, bb) > in.eps_corr ? 1 : 0;
      if (ok) hat = spectral(ab, aa, bb);
    }
    if (chk && b < p && lane == 2) {
      // r_feas_i (Eq. feas_stop)
      const double s2 = a[A_S2];
      double d = 0.0;
      if (bd.type == BT_BOUNDS || bd.type == BT_LINE) {
        d = sqrt(a[A_FEAS_D2]);
      } else if (bd.type == BT_L2) {
        // ||s - P(s)|| = ||s - d|| - sigma outside the ball (d = 0 unless a data fit)
        const double r = bd.bv_lo >= 0 ? sqrt(a[A_FEAS_D2]) : sqrt(s2);
        d = fmax(0.0, r - sc.sigma[b]);
      } else if (bd.type == BT_ANNULUS) {
        const double n = sqrt(s2);  // distance to the nearer sphere; s = 0 stays 0
        d = n > bd.hi ? n - bd.hi : (n > 0.0 && n < bd.lo ? bd.lo - n : 0.0);
      } else {
        const JobScal &js = jscal[bd.job_s];
        if (js.mode == JM_ALL) {
          d = 0.0;
        } else if (js.mode == JM_NONE) {
          d = sqrt(s2);
        } else if (bd.type == BT_L1) {
          // s - P(s) = sign(s) min(|s|, theta)
          d = sqrt(fmax(js.c_above * js.theta * js.theta + (s2 - js.s2_above), 0.0));
        } else {
          // ||s - P(s)||^2 = ||s||^2 - (squares of the k kept entries)
          d = sqrt(fmax(s2 - js.s2_above - (double)js.need * js.kval * js.kval, 0.0));
        }
      }
      fe = s2 > 0.0 ? d / sqrt(s2) : d;
    }
    const bool aok = __shfl_sync(FULL, ok, 0) != 0, bok = __shfl_sync(FULL, ok, 1) != 0;
    const double ah = __shfl_sync(FULL, hat, 0), bh = __shfl_sync(FULL, hat, 1);
    fe = __shfl_sync(FULL, fe, 2);
    if (lane == 0) {
      double rho_b = sc.rho[b], gam_b = sc.gamma[b];
      if (chk && b < p) s_feas[b] = fe;
      if (ad && have_k0) {
        // Algorithm adapt-rho-gamma; the first call only stores the k0
        // quantities (done by the set and final passes)
        double r, g;
        if (aok && bok) {
          r = sqrt(ah * bh);
          g = 1.0 + 2.0 * r / (ah + bh);
        } else if (aok) {
          r = ah;
          g = 1.9;
        } else if (bok) {
          r = bh;
          g = 1.1;
        } else {
          r = rho_b;
          g = 1.5;
        }
        if (in.adapt == 1) g = gam_b;
        rho_b = r;
        gam_b = fmin(g, in.gamma_max);
      }
      s_rho[b] = rho_b;
      s_gam[b] = gam_b;
    }
  }
  __syncthreads();
  if (wid != 0) return;

  // ---- phase 2: warp 0, one lane per block
  const int b = lane;
  // CG steps of this iteration: the state the last step launch stored
  int cg_steps = 0;
  if (cg_launch > 0) {
    const CgState &st = sc.cg[(cg_launch + 1) & 1];
    cg_steps = st.steps + st.active;
  }
  if (b == 0) {
    sc.cg_steps = cg_steps;
    sc.cg_total += cg_steps;
  }
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  double *tr = in.trace ? in.trace + (int64_t)(k - 1) * in.trace_w : nullptr;
  if (tr) {
    if (b < nb) {
      tr[b] = sc.rho[b];
      tr[nb + b] = sc.gamma[b];
    }
    if (b == 0) {
      tr[2 * nb] = cg_steps;
      tr[2 * nb + 1] = nan;
    }
    if (b < p) tr[2 * nb + 2 + b] = chk ? s_feas[b] : nan;
  }
  bool stop = false;
  if (chk) {
    bool ok = true;
    if (b < p) {
      sc.r_feas[b] = s_feas[b];
      ok = s_feas[b] < in.eps_feas;
    }
    const bool all_ok = __all_sync(FULL, ok);
    // r_evol (Eq. obj_stop): max over the stored history
    const int jmax = k < in.hist ? k : in.hist;
    double dmax = (b >= 1 && b <= jmax) ? sc.acc_ring[b] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, o));
    const double xn = sqrt(sc.acc_ring[0]);
    const double r_evol = xn > 0.0 ? sqrt(dmax) / xn : sqrt(dmax);
    if (b == 0) {
      sc.r_evol = r_evol;
      if (tr) tr[2 * nb + 1] = r_evol;
    }
    stop = (in.stop == 1 && all_ok && r_evol < in.eps_evol) || (in.stop == 2 && all_ok);
  }
  if (b == 0) sc.iters = k;
  if (stop) {
    if (b == 0) {
      sc.done = 1;
      sc.stop_reason = 1;
      atomicAdd(in.ndone, 1u);
    }
  } else if ((ad && have_k0) || (in.rho_sched && k < in.max_iter)) {
    // rho / gamma change (an adapt step or a replayed schedule): the block
    // scalars and the stencil coefficients follow
    double rho_b = b < nb ? s_rho[b] : 1.0, gam_b = b < nb ? s_gam[b] : 1.0;
    if (ad && have_k0) {
      // safeguard: rho_i within a factor R of rho_{p+1} (direct form: of 1)
      const double ref = in.alg1 ? __shfl_sync(FULL, rho_b, p) : 1.0;
      const double R = in.rho_ratio_max;
      if (b < p) rho_b = fmin(fmax(rho_b, ref / R), ref * R);
    }
    if (in.rho_sched && k < in.max_iter && b < nb) {
      rho_b = in.rho_sched[(int64_t)k * nb + b];
      if (in.gamma_sched) gam_b = in.gamma_sched[(int64_t)k * nb + b];
    }
    // block scalars per lane; the stencil coefficients of C (Eq. sys_mat)
    // summed by lane 0 in block order, as set_coefficients does
    if (b < nb) {
      sc.rho[b] = rho_b;
      sc.gamma[b] = gam_b;
      sc.irho[b] = __drcp_rn(rho_b);  // = 1 / rho correctly rounded, as the division
      sc.inv1p[b] = __drcp_rn(1.0 + rho_b);
      store_block_f32(sc, b);
      s_rho[b] = rho_b;
    }
    __syncwarp();
    if (b == 0) {
      double c0 = in.alg1 ? 0.0 : 1.0, cz = 0.0, cx = 0.0, cy = 0.0;
      for (int j = 0; j < nb; ++j) {
        const double r = s_rho[j];
        switch (in.blk[j].op) {
          case SIP_OP_I: c0 += r; break;
          case SIP_OP_DZ: cz += r; break;
          case SIP_OP_DX: cx += r; break;
          case SIP_OP_DY: cy += r; break;
          case SIP_OP_BLUR: break;  // rho_F F^T F: the blur term of the CG launches
          default: cz += r; cx += r; if (in.ndim == 3) cy += r; break;
        }
      }
      sc.c0 = c0;
      sc.cz = cz * in.ihz * in.ihz;
      sc.cx = cx * in.ihx * in.ihx;
      sc.cy = cy * in.ihy * in.ihy;
      store_coef_f32(sc);
    }
  }
  if (!stop && b == 0) {
    if (ad) sc.have_k0 = 1;
    sc.k = k + 1;
    if (k >= in.max_iter) {
      sc.done = 1;
      atomicAdd(in.ndone, 1u);
    }
  }
  __syncwarp();
  // top-k selection windows: re-centre on this iteration's k-th value, widen
  // after a miss, narrow after an overflow or a crowded hit; clear the counts
  {
    bool hit = false;
    if (b < nb && in.blk[b].type == BT_CARD && in.blk[b].job_w >= 0) {
      JobScal &js = jscal[in.blk[b].job_w];
      hit = js.win_hit != 0;
      if (in.select_window && js.active && js.mode == JM_SELECT) {
        double r = js.win_rel;
        if (js.win_on) {
          if (hit)
            r = js.win_n > kWinCap / 4 ? 0.5 * r : r;
          else
            r = js.win_n > kWinCap ? 0.25 * r : 2.0 * r;
        }
        r = fmin(fmax(r, kWinRelMin), kWinRelMax);
        const double kv = js.kval;
        js.win_rel = r;
        js.win_on = kv > 0.0 ? 1 : 0;
        js.win_lo = kv * (1.0 - r);
        js.win_hi = kv * (1.0 + r);
      }
      js.win_n = 0;
      js.win_above = 0;
      js.win_hit = 0;
    }
    const unsigned hits = __ballot_sync(FULL, hit);
    if (b == 0 && hits) sc.win_hits += __popc(hits);
  }
  // clear the per-iteration accumulators
  double *acc = &sc.acc[0][0];
  for (int j = b; j < kMaxBlocks * kNAcc; j += 32) acc[j] = 0.0;
  if (b <= kMaxHist) sc.acc_ring[b] = 0.0;
}

__global__ void __launch_bounds__(32 * kTailWarps) k_tail(const InstDev *__restrict__ insts,
                                                          InstScal *__restrict__ scal,
                                                          JobScal *__restrict__ jscal, int ninst,
                                                          int cg_launch, unsigned long long *ts,
                                                          const __grid_constant__ InstOne one) {
  const Stamp stamp(ts);
  if ((int)blockIdx.x >= ninst) return;
  if (one.on) {  // the descriptor is a launch parameter
    body_tail(0, &one.d, scal, jscal, cg_launch);
    return;
  }
  // the tail's scattered descriptor reads (blocks, operators, options) from
  // a shared-memory copy
  __shared__ InstDev s_in;
  static_assert(sizeof(InstDev) % 8 == 0, "InstDev copies in 8-byte words");
  const uint2 *src = reinterpret_cast<const uint2 *>(&insts[blockIdx.x]);
  uint2 *dst = reinterpret_cast<uint2 *>(&s_in);
  for (int i = threadIdx.x; i < (int)(sizeof(InstDev) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  body_tail(0, &s_in, scal + blockIdx.x, jscal, cg_launch);
}

// --------------------------------------------------------------------------
// Persistent form: every phase of the iteration in one cooperative launch.
// Kernel boundaries become grid barriers; the work items and the phase
// bodies are the ones of the separate kernels above.
// --------------------------------------------------------------------------
// Barrier words: [0] arrivals, [1] generation, [2] error, [3] unused.
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed polls of barrier words (an acquire load per poll would also cost
// the SM's other CTAs their L1 contents); the waits fence once afterwards.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier with a bounded wait.  A CTA that waits longer than
// kBarrierSpins polls (seconds) records SIP_ERR_TIMEOUT in bar[2] and every
// CTA returns false, so the kernel ends instead of hanging.
constexpr long long kBarrierSpins = 1ll << 26;
__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t expected, long long max_spins) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const uint32_t g = ld_acquire(&bar[1]);
    __threadfence();
    const uint32_t arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == expected) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long spins = 0;
      while (ld_relaxed(&bar[1]) == g) {
        if (ld_relaxed(&bar[2]) != 0 || ++spins > max_spins) {
          atomicExch(&bar[2], (uint32_t)SIP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ld_acquire(&bar[2]) != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// dynamic shared memory of the persistent kernel: the select histogram or
// the per-line arrays, whichever is larger
template <typename T>
constexpr size_t fused_smem() {
  return BinAcc<T>::kSmem > line_smem<T>() ? BinAcc<T>::kSmem : line_smem<T>();
}

struct FusedArgs {
  const Tile *tn, *tset, *tsel, *tfin, *tline;
  int nt_n, nt_set, nt_sel, nt_fin, nt_line;
  const InstDev *insts;
  InstScal *scal;
  const JobDev *jobs;
  JobScal *jscal;
  uint32_t *hcnt;
  double *hs1, *hs2, *hs3;
  int64_t hstride;
  uint32_t *ties;
  uint32_t *bar;
  const uint32_t *ndone;
  int ninst, npass, cg_launch, any_card, any_fin, iters;
  uint32_t bar_expected;  // arrivals per barrier: the grid (plus a test hook's extra)
  long long bar_spins;    // polls before a barrier gives up
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_fused(const FusedArgs A) {
  for (int it = 0; it < A.iters; ++it) {
    for (int i = blockIdx.x; i < A.nt_n; i += gridDim.x) body_rhs<T>(A.tn[i], A.insts, A.scal);
    if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    for (int i = blockIdx.x; i < A.nt_n; i += gridDim.x) body_cg_w0<T>(A.tn[i], A.insts, A.scal);
    if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    for (int j = 0; j < A.cg_launch; ++j) {
      for (int i = blockIdx.x; i < A.nt_n; i += gridDim.x) body_cg_step<T>(A.tn[i], A.insts, A.scal, 2 + j);
      if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    }
    for (int i = blockIdx.x; i < A.nt_set; i += gridDim.x) body_setpass<T>(A.tset[i], A.insts, A.scal, A.jscal, A.jobs);
    if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    if (A.nt_sel) {
      for (int pass = 0; pass < A.npass; ++pass) {
        for (int i = blockIdx.x; i < A.nt_sel; i += gridDim.x)
          body_select<T>(A.tsel[i], A.insts, A.scal, A.jobs, A.jscal, A.hcnt, A.hs1, A.hs2, A.hs3, A.hstride, pass);
        if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
      }
    }
    if (A.any_card) {
      for (int i = blockIdx.x; i < A.nt_fin; i += gridDim.x) body_ties<T>(A.tfin[i], A.insts, A.scal, A.jobs, A.jscal, A.ties);
      if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    }
    if (A.nt_line) {
      extern __shared__ unsigned char smem_raw[];
      for (int i = blockIdx.x; i < A.nt_line; i += gridDim.x) body_lines<T>(A.tline[i], A.insts, A.scal, smem_raw);
      if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    }
    if (A.any_fin) {
      for (int i = blockIdx.x; i < A.nt_fin; i += gridDim.x) body_final<T>(A.tfin[i], A.insts, A.scal, A.jobs, A.jscal, A.ties);
      if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    }
    for (int i = blockIdx.x; i < A.ninst; i += gridDim.x) body_tail(i, A.insts, A.scal, A.jscal, A.cg_launch);
    if (!grid_barrier(A.bar, A.bar_expected, A.bar_spins)) return;
    if (ld_acquire(A.ndone) >= (uint32_t)A.ninst) return;  // every instance stopped
  }
}

// Cluster form of the iteration: the same phase bodies, one thread-block
// cluster per instance.  The cluster's CTAs walk the instance's own work
// items (rank r takes items r, r + C, ...) and meet at the cluster's
// hardware barrier between phases instead of at a kernel boundary or a
// software grid barrier; every phase's data stays in L2.  A cluster runs its
// instance until the instance stops (max_iter or the stopping rule), then
// takes the next one (cid, cid + clusters, ...).  No wait here can outlast
// the cluster's own progress: the barrier completes once every CTA of the
// cluster arrives, and every CTA runs the same sequence of phases.
// The barrier's arrive has release and its wait acquire semantics at
// cluster scope: every CTA's global writes of a phase are visible to the
// cluster's CTAs in the next.
__device__ __forceinline__ void cluster_phase_sync() { cooperative_groups::this_cluster().sync(); }

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_fused_cluster(const FusedArgs A) {
  namespace cg = cooperative_groups;
  const cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int r = (int)cl.block_rank();
  const int ncl = (int)(gridDim.x / C);
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_done;
  for (int inst = (int)(blockIdx.x / C); inst < A.ninst; inst += ncl) {
    const InstDev &in = A.insts[inst];
    const int tn0 = in.tn0, tn1 = in.tn0 + in.nt_n;
    const int ts0 = in.tset0, ts1 = in.tset0 + in.nt_set;
    const int tq0 = in.tsel0, tq1 = in.tsel0 + in.nt_sel;
    const int tf0 = in.tfin0, tf1 = in.tfin0 + in.nt_fin;
    const int tl0 = in.tline0, tl1 = in.tline0 + in.nt_line;
    bool has_card = false, has_fin = in.nt_fin > 0;
    for (int b = 0; b < in.nb; ++b) has_card = has_card || in.blk[b].type == BT_CARD;
    for (int it = 0; it < A.iters; ++it) {
      for (int i = tn0 + r; i < tn1; i += C) body_rhs<T>(A.tn[i], A.insts, A.scal);
      cluster_phase_sync();
      for (int i = tn0 + r; i < tn1; i += C) body_cg_w0<T>(A.tn[i], A.insts, A.scal);
      cluster_phase_sync();
      for (int j = 0; j < A.cg_launch; ++j) {
        for (int i = tn0 + r; i < tn1; i += C) body_cg_step<T>(A.tn[i], A.insts, A.scal, 2 + j);
        cluster_phase_sync();
      }
      for (int i = ts0 + r; i < ts1; i += C) body_setpass<T>(A.tset[i], A.insts, A.scal, A.jscal, A.jobs);
      cluster_phase_sync();
      if (tq1 > tq0) {
        for (int pass = 0; pass < A.npass; ++pass) {
          for (int i = tq0 + r; i < tq1; i += C)
            body_select<T>(A.tsel[i], A.insts, A.scal, A.jobs, A.jscal, A.hcnt, A.hs1, A.hs2, A.hs3, A.hstride, pass);
          cluster_phase_sync();
        }
      }
      if (has_card) {
        for (int i = tf0 + r; i < tf1; i += C) body_ties<T>(A.tfin[i], A.insts, A.scal, A.jobs, A.jscal, A.ties);
        cluster_phase_sync();
      }
      if (tl1 > tl0) {
        for (int i = tl0 + r; i < tl1; i += C) body_lines<T>(A.tline[i], A.insts, A.scal, smem_raw);
        cluster_phase_sync();
      }
      if (has_fin) {
        for (int i = tf0 + r; i < tf1; i += C) body_final<T>(A.tfin[i], A.insts, A.scal, A.jobs, A.jscal, A.ties);
        cluster_phase_sync();
      }
      if (r == 0) body_tail(inst, A.insts, A.scal, A.jscal, A.cg_launch);
      cluster_phase_sync();
      // the tail's stop decision, read by every CTA after the barrier: the
      // whole cluster leaves the instance together
      if (threadIdx.x == 0) s_done = ld_acquire((const uint32_t *)&A.scal[inst].done) != 0u;
      __syncthreads();
      if (s_done) break;
    }
  }
}

}  // namespace sip

// ==========================================================================
// Per-call set-up: scalars, relative radii, non-finite model check.
// ==========================================================================
namespace sip {

__global__ void k_init(const InstDev *__restrict__ insts, InstScal *__restrict__ scal, JobScal *__restrict__ jscal,
                       int ninst) {
  const int i = blockIdx.x;
  if (i >= ninst) return;
  const InstDev &in = insts[i];
  InstScal &sc = scal[i];
  double *acc = &sc.acc[0][0];
  for (int j = threadIdx.x; j < kMaxBlocks * kNAcc; j += blockDim.x) acc[j] = 0.0;
  for (int j = threadIdx.x; j <= kMaxHist; j += blockDim.x) sc.acc_ring[j] = 0.0;
  if (threadIdx.x != 0) return;
  sc.k = 1;
  sc.done = 0;
  sc.iters = 0;
  sc.stop_reason = 0;
  sc.cg_steps = 0;
  sc.cg_total = 0;
  sc.have_k0 = 0;
  sc.nonfinite = 0;
  sc.cnt_set = sc.cnt_norm = 0;
  sc.win_hits = 0;
  for (int j = 0; j < in.njob; ++j) {  // selection windows start closed
    JobScal &js = jscal[in.job0 + j];
    js.win_on = js.win_hit = 0;
    js.win_n = 0;
    js.win_above = 0;
    js.win_lo = js.win_hi = 0.0;
    js.win_rel = kWinRel0;
  }
  for (int j = 0; j < 2; ++j) sc.cg[j] = CgState{0.0, 0.0, 0.0, 0.f, 0.f, 0.f, 0, 0};
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int b = 0; b < kMaxSets; ++b) sc.r_feas[b] = nan;
  sc.r_evol = nan;
  for (int b = 0; b < in.nb; ++b) {
    sc.rho[b] = in.rho_sched ? in.rho_sched[b] : in.rho0;
    sc.gamma[b] = in.gamma_sched ? in.gamma_sched[b] : in.gamma0;
    sc.l2scale[b] = 1.0;
    sc.sigma[b] = in.blk[b].sigma_abs;
    sc.kcard[b] = in.blk[b].k_abs;
  }
  set_coefficients(in, sc);
}

// Starting rho_i, gamma_i of a warm start written over the initialised
// rho0 / gamma0 values, with every derived scalar (1/rho, 1/(1+rho), C's
// stencil coefficients, the binary32 copies) formed by the same device code
// as after an adapt-rho-gamma call.  One thread.
__global__ void k_load_penalties(const InstDev *__restrict__ insts, InstScal *__restrict__ scal, Penalties pen) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const InstDev &in = insts[0];
  InstScal &sc = scal[0];
  for (int b = 0; b < in.nb; ++b) {
    sc.rho[b] = pen.rho[b];
    sc.gamma[b] = pen.gamma[b];
    sc.l2scale[b] = 1.0;
  }
  set_coefficients(in, sc);
}
cudaError_t launch_load_penalties(cudaStream_t st, const InstDev *insts, InstScal *scal, const Penalties &pen) {
  k_load_penalties<<<1, 32, 0, st>>>(insts, scal, pen);
  return cudaGetLastError();
}

// ||A_i m|| for sets with relative radii, and a finiteness check of m.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_norms(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                    InstScal *__restrict__ scal) {
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  const SegDev sg = in.seg[tl.item];
  const T *__restrict__ m = (const T *)in.m;
  double acc[2] = {0.0, 0.0};
  for (int64_t row = tl.start + threadIdx.x; row < tl.start + tl.len; row += kThreads) {
    if (sg.kind == SEG_RING) {
      if (!isfinite((double)m[row])) acc[0] += 1.0;
    } else {
      int64_t g;
      const double s = (double)seg_forward<T>(in, sg.kind, m, row, g);
      acc[0] += fabs(s);
      acc[1] += s * s;
    }
  }
  block_sum<2>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    if (sg.kind == SEG_RING) {
      if (acc[0] > 0.0) atomicAdd(&sc.nonfinite, 1);
    } else {
      atomicAdd(&sc.acc[sg.block][A_M1], acc[0]);
      atomicAdd(&sc.acc[sg.block][A_M2], acc[1]);
    }
    last = arrive_last(&sc.cnt_norm, (uint32_t)in.nt_set);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  for (int b = 0; b < in.nb; ++b) {
    const BlockDev &bd = in.blk[b];
    if (bd.sigma_rel > 0.0) {
      const double n1 = ldv(&sc.acc[b][A_M1]), n2 = ldv(&sc.acc[b][A_M2]);
      sc.sigma[b] = bd.sigma_rel * (bd.type == BT_L1 ? n1 : sqrt(n2));
    }
    if (bd.k_frac > 0.0) sc.kcard[b] = (int64_t)floor(bd.k_frac * (double)(bd.type == BT_LINE ? bd.line_len : in.N));
    sc.acc[b][A_M1] = 0.0;
    sc.acc[b][A_M2] = 0.0;
  }
  if (*(volatile int *)&sc.nonfinite) {
    sc.done = 1;
    sc.stop_reason = -1;
    atomicAdd(in.ndone, 1u);
  }
}

}  // namespace sip

// ==========================================================================
// Single-step operators (the loop's stencil code on caller buffers)
// ==========================================================================
namespace sip {

// s = A x: thread per output row; in.seg[0..nseg) are the operator's parts
// in row order (row0 = offset of each part).
template <typename T>
__global__ void k_apply_op(const InstDev *__restrict__ inp, const T *__restrict__ x, T *__restrict__ s, int64_t rows) {
  const InstDev &in = *inp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    int sgi = 0;
    while (sgi + 1 < in.nseg && i >= in.seg[sgi + 1].row0) ++sgi;
    int64_t g;
    s[i] = seg_forward<T>(in, in.seg[sgi].kind, x, i - in.seg[sgi].row0, g);
  }
}

template <typename T>
__global__ void k_apply_op_t(const InstDev *__restrict__ inp, const T *__restrict__ s, T *__restrict__ x, int64_t n) {
  const InstDev &in = *inp;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const GridPos p = grid_pos(in, g);
    T acc = T(0);
    for (int sgi = 0; sgi < in.nseg; ++sgi) {
      const int64_t base = in.seg[sgi].row0;
      acc += seg_adjoint<T>(in, in.seg[sgi].kind, p, g, [&](int64_t row) { return s[base + row]; });
    }
    x[g] = acc;
  }
}

template <typename T>
__global__ void k_system_apply(const InstDev *__restrict__ inp, const InstScal *__restrict__ scp,
                               const T *__restrict__ x, T *__restrict__ out, int64_t n) {
  const InstDev &in = *inp;
  const InstScal &sc = *scp;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const GridPos p = grid_pos(in, g);
    out[g] = csys<T>(in, sc, p, g, [&](int64_t i) { return x[i]; });
  }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
// by storage type and by whether the descriptor is a launch parameter
#define SIP_DISPATCH_ONE(L, ONEP, KERNEL, GRID, BLOCK, SMEM, ...)                                   \
  do {                                                                                            \
    if ((L).dtype == SIP_F64) {                                                                   \
      if ((ONEP).on)                                                                              \
        KERNEL<double, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);              \
      else                                                                                        \
        KERNEL<double, false><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);             \
    } else {                                                                                      \
      if ((ONEP).on)                                                                              \
        KERNEL<float, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);               \
      else                                                                                        \
        KERNEL<float, false><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);              \
    }                                                                                             \
  } while (0)

// ... and by whether the plan has a blur block (kernels with the F^T F term)
#define SIP_DISPATCH_ONE_BL(L, ONEP, KERNEL, GRID, BLOCK, SMEM, ...)                             \
  do {                                                                                          \
    if ((L).blur) {                                                                             \
      if ((L).dtype == SIP_F64) {                                                               \
        if ((ONEP).on)                                                                          \
          KERNEL<double, true, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);     \
        else                                                                                    \
          KERNEL<double, false, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);    \
      } else {                                                                                  \
        if ((ONEP).on)                                                                          \
          KERNEL<float, true, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);      \
        else                                                                                    \
          KERNEL<float, false, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);     \
      }                                                                                         \
    } else {                                                                                    \
      SIP_DISPATCH_ONE(L, ONEP, KERNEL, GRID, BLOCK, SMEM, __VA_ARGS__);                        \
    }                                                                                           \
  } while (0)
#define SIP_DISPATCH_BL(L, KERNEL, GRID, BLOCK, SMEM, ...)                                        \
  do {                                                                                          \
    if ((L).dtype == SIP_F64) {                                                                 \
      if ((L).blur)                                                                             \
        KERNEL<double, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);             \
      else                                                                                      \
        KERNEL<double, false><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);            \
    } else {                                                                                    \
      if ((L).blur)                                                                             \
        KERNEL<float, true><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);              \
      else                                                                                      \
        KERNEL<float, false><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);             \
    }                                                                                           \
  } while (0)

#define SIP_DISPATCH(L, KERNEL, GRID, BLOCK, SMEM, ...)                          \
  do {                                                                           \
    if ((L).dtype == SIP_F64)                                                    \
      KERNEL<double><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);     \
    else                                                                         \
      KERNEL<float><<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);      \
  } while (0)

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_init(const Launch &L, const InstDev *insts, InstScal *scal, JobScal *jscal, int ninst) {
  k_init<<<ninst, 32, 0, L.stream>>>(insts, scal, jscal, ninst);
  return cudaGetLastError();
}
cudaError_t launch_norms(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal) {
  SIP_DISPATCH(L, k_norms, nt, kThreads, 0, tiles, insts, scal);
  return cudaGetLastError();
}
cudaError_t launch_rhs(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                       const InstOne &one) {
  SIP_DISPATCH_ONE_BL(L, one, k_rhs, nt, kThreads, 0, tiles, insts, scal, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_rhs_tma(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                           size_t smem, const InstOne &one) {
  if (one.on)
    k_rhs_tma<true><<<nt, kThreads, smem, L.stream>>>(tiles, insts, scal, L.ts, one);
  else
    k_rhs_tma<false><<<nt, kThreads, smem, L.stream>>>(tiles, insts, scal, L.ts, one);
  return cudaGetLastError();
}
int rhs_tma_occupancy(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rhs_tma<false>, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
cudaError_t launch_cg_w0(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const CgOne &one) {
  SIP_DISPATCH_BL(L, k_cg_w0, nt, kThreads, 0, tiles, insts, scal, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_cg_step(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, int ph,
                           const CgOne &one) {
  if (ph == 2)
    SIP_DISPATCH_BL(L, k_cg_first, nt, kThreads, 0, tiles, insts, scal, ph, L.ts, one);
  else
    SIP_DISPATCH_BL(L, k_cg_step, nt, kThreads, 0, tiles, insts, scal, ph, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_cg_last(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, int ph,
                           const CgOne &one) {
  SIP_DISPATCH(L, k_cg_last, nt, kThreads, 0, tiles, insts, scal, ph, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_blur_rhs(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, const InstScal *scal) {
  SIP_DISPATCH(L, k_blur_rhs, nt, kThreads, 0, tiles, insts, scal, L.ts);
  return cudaGetLastError();
}
cudaError_t launch_blur_fwd(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, const InstScal *scal) {
  SIP_DISPATCH(L, k_blur_fwd, nt, kThreads, 0, tiles, insts, scal, L.ts);
  return cudaGetLastError();
}
cudaError_t launch_cg_step_blur(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                                int ph) {
  SIP_DISPATCH(L, k_cg_step_blur, nt, kThreads, 0, tiles, insts, scal, ph, L.ts);
  return cudaGetLastError();
}
cudaError_t launch_setpass(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                           JobScal *jscal, const JobDev *jobs, const InstOne &one) {
  SIP_DISPATCH_ONE_BL(L, one, k_setpass, nt, kThreads, 0, tiles, insts, scal, jscal, jobs, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_select(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                          const JobDev *jobs, JobScal *jscal, uint32_t *hcnt, double *hs1, double *hs2, double *hs3,
                          int64_t hstride, int pass, const InstOne &one) {
  SIP_DISPATCH_ONE(L, one, k_select, nt, kThreads, (L.dtype == SIP_F64 ? BinAcc<double>::kSmem : BinAcc<float>::kSmem),
                   tiles, insts, scal, jobs, jscal, hcnt, hs1, hs2, hs3, hstride, pass, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_lines(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const InstOne &one) {
  SIP_DISPATCH_ONE(L, one, k_lines, nt, kThreads, (L.dtype == SIP_F64 ? line_smem<double>() : line_smem<float>()), tiles, insts,
               scal, L.ts, one);
  return cudaGetLastError();
}
// Parallel Dykstra sweep update (Appendix A): with y_i = P_i(v_i) packed in
// y (instance i at i * n), x = sum_i w_i y_i and v_i = x + v_i - y_i (v packed
// the same way, updated in place).
template <typename T>
__global__ void k_dykstra_update(const T *__restrict__ y, T *__restrict__ v, T *__restrict__ x, int p, int64_t n) {
  const T wgt = T(1) / T(p);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int i = 0; i < p; ++i) acc += wgt * y[(int64_t)i * n + g];
    x[g] = acc;
    for (int i = 0; i < p; ++i) v[(int64_t)i * n + g] = acc + v[(int64_t)i * n + g] - y[(int64_t)i * n + g];
  }
}
// BF16 storage trial: round n binary32 values in place to bfloat16.
__global__ void k_round_bf16(float *__restrict__ a, int64_t n) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    a[g] = rbf(a[g]);
}
cudaError_t launch_round_bf16(const Launch &L, void *a, int64_t n) {
  if (n <= 0 || L.dtype != SIP_F32) return cudaSuccess;
  k_round_bf16<<<grid_for(n), 256, 0, L.stream>>>((float *)a, n);
  return cudaGetLastError();
}
cudaError_t launch_dykstra_update(const Launch &L, const void *y, void *v, void *x, int p, int64_t n) {
  if (L.dtype == SIP_F64)
    k_dykstra_update<double><<<grid_for(n), 256, 0, L.stream>>>((const double *)y, (double *)v, (double *)x, p, n);
  else
    k_dykstra_update<float><<<grid_for(n), 256, 0, L.stream>>>((const float *)y, (float *)v, (float *)x, p, n);
  return cudaGetLastError();
}

cudaError_t kernels_setup() {
  // the binary32 select histogram needs 56 KB of shared memory: opt in once
  // per device (a function attribute belongs to the current device's context)
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_select<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BinAcc<float>::kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_select<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BinAcc<double>::kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rhs_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRhsSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lines<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lines<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_select<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BinAcc<float>::kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_select<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BinAcc<double>::kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rhs_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRhsSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lines<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lines<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused_cluster<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused_cluster<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_smem<double>());
  if (e != cudaSuccess) return e;
  // clusters of 16 CTAs are beyond the portable limit of 8
  e = cudaFuncSetAttribute(k_fused_cluster<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fused_cluster<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

// CTAs per SM of the kernels that share one work-item list.
int launch_occupancy(int dtype, int kind) {
  int n = 0, best = 1 << 30;
  auto occ = [&](const void *f, size_t smem) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) == cudaSuccess && n > 0 && n < best)
      best = n;
  };
  const bool d = dtype == SIP_F64;
  switch (kind) {
    case 0:  // grid-point items: rhs, CG
      occ(d ? (const void *)k_rhs<double, false> : (const void *)k_rhs<float, false>, 0);
      occ(d ? (const void *)k_cg_w0<double> : (const void *)k_cg_w0<float>, 0);
      occ(d ? (const void *)k_cg_step<double> : (const void *)k_cg_step<float>, 0);
      break;
    case 1:  // segment items: set pass
      occ(d ? (const void *)k_setpass<double, false> : (const void *)k_setpass<float, false>, 0);
      break;
    case 2:  // selection items
      occ(d ? (const void *)k_select<double, false> : (const void *)k_select<float, false>,
          d ? BinAcc<double>::kSmem : BinAcc<float>::kSmem);
      break;
    case 4:  // per-line items
      occ(d ? (const void *)k_lines<double, false> : (const void *)k_lines<float, false>, d ? line_smem<double>() : line_smem<float>());
      break;
    default:  // final-pass items
      occ(d ? (const void *)k_final<double, false> : (const void *)k_final<float, false>, 0);
      occ(d ? (const void *)k_ties<double, false> : (const void *)k_ties<float, false>, 0);
      break;
  }
  cudaGetLastError();
  return best == (1 << 30) ? 1 : best;
}

static FusedArgs fused_args(const Launch &L, const FusedLaunch &F) {
  FusedArgs A;
  A.tn = F.tn;
  A.tset = F.tset;
  A.tsel = F.tsel;
  A.tfin = F.tfin;
  A.tline = F.tline;
  A.nt_line = F.nt_line;
  A.nt_n = F.nt_n;
  A.nt_set = F.nt_set;
  A.nt_sel = F.nt_sel;
  A.nt_fin = F.nt_fin;
  A.insts = F.insts;
  A.scal = F.scal;
  A.jobs = F.jobs;
  A.jscal = F.jscal;
  A.hcnt = F.hcnt;
  A.hs1 = F.hs1;
  A.hs2 = F.hs2;
  A.hs3 = F.hs3;
  A.hstride = F.hstride;
  A.ties = F.ties;
  A.bar = F.bar;
  A.ndone = F.ndone;
  A.ninst = F.ninst;
  A.npass = select_passes(L.dtype);
  A.cg_launch = F.cg_launch;
  A.any_card = F.any_card;
  A.any_fin = F.any_fin;
  A.iters = F.iters;
  A.bar_expected = 0;
  A.bar_spins = kBarrierSpins;
  return A;
}

static cudaLaunchConfig_t cluster_config(int dtype, int clusters, int csize, cudaStream_t st,
                                         cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * csize), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = dtype == SIP_F64 ? fused_smem<double>() : fused_smem<float>();
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t launch_fused_cluster(const Launch &L, const FusedLaunch &F, int clusters, int csize) {
  const FusedArgs A = fused_args(L, F);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(L.dtype, clusters, csize, L.stream, attr);
  if (L.dtype == SIP_F64) return cudaLaunchKernelEx(&cfg, k_fused_cluster<double>, A);
  return cudaLaunchKernelEx(&cfg, k_fused_cluster<float>, A);
}

int fused_cluster_capacity(int dtype, int csize) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(dtype, 1, csize, nullptr, attr);
  int n = 0;
  const cudaError_t e = dtype == SIP_F64
                            ? cudaOccupancyMaxActiveClusters(&n, (const void *)k_fused_cluster<double>, &cfg)
                            : cudaOccupancyMaxActiveClusters(&n, (const void *)k_fused_cluster<float>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_fused(const Launch &L, const FusedLaunch &F, int grid) {
  FusedArgs A = fused_args(L, F);
  A.bar_expected = (uint32_t)grid + F.bar_extra;
  A.bar_spins = F.bar_spins > 0 ? F.bar_spins : kBarrierSpins;
  void *args[] = {&A};
  const bool d = L.dtype == SIP_F64;
  const size_t smem = d ? fused_smem<double>() : fused_smem<float>();
  return cudaLaunchCooperativeKernel(d ? (const void *)k_fused<double> : (const void *)k_fused<float>, grid, kThreads,
                                     args, smem, L.stream);
}

// CTAs of the persistent kernel that are resident at once (its cooperative grid).
int fused_grid(int dtype) {
  int dev = 0, sms = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool d = dtype == SIP_F64;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d ? (const void *)k_fused<double> : (const void *)k_fused<float>,
                                                kThreads, d ? fused_smem<double>() : fused_smem<float>());
  cudaGetLastError();
  return sms * n;
}

int select_passes(int dtype) { return dtype == SIP_F64 ? num_passes<double>() : num_passes<float>(); }
cudaError_t launch_ties(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                        const JobDev *jobs, JobScal *jscal, uint32_t *ties, const InstOne &one) {
  SIP_DISPATCH_ONE(L, one, k_ties, nt, kThreads, 0, tiles, insts, scal, jobs, jscal, ties, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_final(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const JobDev *jobs, const JobScal *jscal, const uint32_t *ties, const InstOne &one) {
  SIP_DISPATCH_ONE(L, one, k_final, nt, kThreads, 0, tiles, insts, scal, jobs, jscal, ties, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_tail(const Launch &L, const InstDev *insts, InstScal *scal, JobScal *jscal, int ninst,
                        int cg_launch, const InstOne &one) {
  k_tail<<<ninst, 32 * kTailWarps, 0, L.stream>>>(insts, scal, jscal, ninst, cg_launch, L.ts, one);
  return cudaGetLastError();
}
cudaError_t launch_apply_op(const Launch &L, const InstDev *in, const void *x, void *s, int64_t rows) {
  if (L.dtype == SIP_F64)
    k_apply_op<double><<<grid_for(rows), 256, 0, L.stream>>>(in, (const double *)x, (double *)s, rows);
  else
    k_apply_op<float><<<grid_for(rows), 256, 0, L.stream>>>(in, (const float *)x, (float *)s, rows);
  return cudaGetLastError();
}
cudaError_t launch_apply_op_t(const Launch &L, const InstDev *in, const void *s, void *x, int64_t n) {
  if (L.dtype == SIP_F64)
    k_apply_op_t<double><<<grid_for(n), 256, 0, L.stream>>>(in, (const double *)s, (double *)x, n);
  else
    k_apply_op_t<float><<<grid_for(n), 256, 0, L.stream>>>(in, (const float *)s, (float *)x, n);
  return cudaGetLastError();
}
cudaError_t launch_system_apply(const Launch &L, const InstDev *in, const InstScal *sc, const void *x, void *out,
                                int64_t n) {
  if (L.dtype == SIP_F64)
    k_system_apply<double><<<grid_for(n), 256, 0, L.stream>>>(in, sc, (const double *)x, (double *)out, n);
  else
    k_system_apply<float><<<grid_for(n), 256, 0, L.stream>>>(in, sc, (const float *)x, (float *)out, n);
  return cudaGetLastError();
}

}  // namespace sip
