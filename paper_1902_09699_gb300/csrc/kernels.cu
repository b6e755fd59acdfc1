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
// All scalars live on the device; reductions are binary64 and finish in the
// last CTA to arrive ("last tile"), so no launch depends on a host sync.
#include <cstdint>
#include <cuda_runtime.h>
#include <math.h>

#include "sip_dev.cuh"
#include "sip_kernels.h"

namespace sip {

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ double ldv(const double *p) { return *(const volatile double *)p; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums NQ values over the CTA; thread 0 gets the totals.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ]) {
  __shared__ double sm[NQ][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double t = warp_sum(v[q]);
    if (lane == 0) sm[q][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double t = lane < kThreads / 32 ? sm[q][lane] : 0.0;
      v[q] = warp_sum(t);
    }
  }
  __syncthreads();
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

__device__ __forceinline__ bool adapt_iter(const InstDev &in, int k) {
  return in.adapt != 0 && in.rho_sched == nullptr &&
         (k % in.adapt_every) == (1 % in.adapt_every);
}
__device__ __forceinline__ bool check_iter(const InstDev &in, int k) { return (k % in.check_every) == 0; }

// s = A x for one row of a segment (Eq. FD_mat): forward differences scaled
// by 1/h, no boundary rows.  g receives the grid index of the row's base
// sample.
template <typename T>
__device__ __forceinline__ T seg_forward(const InstDev &in, int kind, const T *__restrict__ x,
                                         int64_t row, int64_t &g) {
  switch (kind) {
    case SEG_DZ: {
      const uint32_t r = (uint32_t)row, d = (uint32_t)(in.nz - 1);
      const uint32_t t = r / d;             // ix + nx*iy
      g = (int64_t)r + t;                   // iz + nz*t
      return (x[g + 1] - x[g]) * (T)in.ihz;
    }
    case SEG_DX: {
      const uint32_t r = (uint32_t)row, nz = (uint32_t)in.nz;
      const uint32_t t = r / nz;            // ix + (nx-1)*iy
      const uint32_t iy = t / (uint32_t)(in.nx - 1);
      g = (int64_t)r + (int64_t)nz * iy;
      return (x[g + nz] - x[g]) * (T)in.ihx;
    }
    case SEG_DY: {
      g = row;
      return (x[g + (int64_t)in.nz * in.nx] - x[g]) * (T)in.ihy;
    }
    default:
      g = row;
      return x[row];
  }
}

struct GridPos {
  int32_t iz, ix, iy;
  int64_t t;  // ix + nx*iy
};
__device__ __forceinline__ GridPos grid_pos(const InstDev &in, int64_t g) {
  GridPos p;
  const uint32_t gg = (uint32_t)g, nz = (uint32_t)in.nz;
  const uint32_t t = gg / nz;
  p.iz = (int32_t)(gg - t * nz);
  p.t = t;
  const uint32_t iy = t / (uint32_t)in.nx;
  p.iy = (int32_t)iy;
  p.ix = (int32_t)(t - iy * (uint32_t)in.nx);
  return p;
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
      return (a - b) * (T)in.ihz;
    }
    case SEG_DX: {
      const int64_t r = g - (int64_t)in.nz * p.iy;  // iz + nz*(ix + (nx-1)*iy)
      T a = p.ix >= 1 ? u(r - in.nz) : T(0);
      T b = p.ix <= in.nx - 2 ? u(r) : T(0);
      return (a - b) * (T)in.ihx;
    }
    case SEG_DY: {
      const int64_t s = (int64_t)in.nz * in.nx;
      T a = p.iy >= 1 ? u(g - s) : T(0);
      T b = p.iy <= in.ny - 2 ? u(g) : T(0);
      return (a - b) * (T)in.ihy;
    }
    default:
      return u(g);
  }
}

// (C v)[g] with C = c0 I + cz D_z^T D_z + cx D_x^T D_x + cy D_y^T D_y
// (Eq. sys_mat); D^T D along an axis is the Neumann second difference.
template <typename T, typename V>
__device__ __forceinline__ T csys(const InstDev &in, const InstScal &sc, const GridPos &p, int64_t g, V v) {
  const T c = v(g);
  T lz = T(0), lx = T(0), ly = T(0);
  if (p.iz > 0) lz += c - v(g - 1);
  if (p.iz < in.nz - 1) lz += c - v(g + 1);
  if (p.ix > 0) lx += c - v(g - in.nz);
  if (p.ix < in.nx - 1) lx += c - v(g + in.nz);
  if (in.ny > 1) {
    const int64_t s = (int64_t)in.nz * in.nx;
    if (p.iy > 0) ly += c - v(g - s);
    if (p.iy < in.ny - 1) ly += c - v(g + s);
  }
  return (T)sc.c0 * c + (T)sc.cz * lz + (T)sc.cx * lx + (T)sc.cy * ly;
}

// --------------------------------------------------------------------------
// x-update right-hand side and warm residual
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rhs(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                  InstScal *__restrict__ scal) {
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  const T *__restrict__ x = (const T *)in.x;
  const T *__restrict__ y = (const T *)in.y;
  const T *__restrict__ v = (const T *)in.v;
  const T *__restrict__ m = (const T *)in.m;
  T *__restrict__ r = (T *)in.r;
  double acc[2] = {0.0, 0.0};
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t g = tl.start + threadIdx.x + (int64_t)e * kThreads;
    if (g >= tl.start + tl.len) break;
    const GridPos p = grid_pos(in, g);
    T b = in.alg1 ? T(0) : m[g];
    for (int sgi = 0; sgi < in.nseg; ++sgi) {
      const SegDev &sg = in.seg[sgi];
      if (sg.kind == SEG_RING) continue;
      const int blk = sg.block;
      const T rho = (T)sc.rho[blk];
      const int64_t base = in.blk[blk].yoff + sg.row0;
      b += seg_adjoint<T>(in, sg.kind, p, g, [&](int64_t row) { return rho * y[base + row] + v[base + row]; });
    }
    const T cx = csys<T>(in, sc, p, g, [&](int64_t i) { return x[i]; });
    const T rv = b - cx;
    r[g] = rv;
    acc[0] += (double)b * (double)b;
    acc[1] += (double)rv * (double)rv;
  }
  block_sum<2>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    atomicAdd(&sc.acc_n[0], acc[0]);
    atomicAdd(&sc.acc_n[1], acc[1]);
    last = arrive_last(&sc.cnt_n, (uint32_t)in.nt_n);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    const double bn = ldv(&sc.acc_n[0]), rr = ldv(&sc.acc_n[1]);
    sc.acc_n[0] = 0.0;
    sc.acc_n[1] = 0.0;
    sc.bnorm2 = bn;
    sc.rr = rr;
    sc.rr0 = rr;
    sc.beta = 0.0;
    sc.cg_steps = 0;
    const int limit = in.cg_iters > 0 ? in.cg_iters : in.cg_max;
    sc.cg_active = (limit > 0 && rr > 0.0) ? 1 : 0;
  }
}

// --------------------------------------------------------------------------
// CG: direction + matrix-vector product
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_dir(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                     InstScal *__restrict__ scal) {
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done || !sc.cg_active) return;
  const T *__restrict__ r = (const T *)in.r;
  const T *__restrict__ pold = (const T *)(sc.pbuf ? in.p1 : in.p0);
  T *__restrict__ pnew = (T *)(sc.pbuf ? in.p0 : in.p1);
  T *__restrict__ q = (T *)in.q;
  const bool first = sc.cg_steps == 0;
  const T beta = (T)sc.beta;
  double acc[1] = {0.0};
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t g = tl.start + threadIdx.x + (int64_t)e * kThreads;
    if (g >= tl.start + tl.len) break;
    const GridPos p = grid_pos(in, g);
    T pg, qg;
    if (first) {
      pg = r[g];
      qg = csys<T>(in, sc, p, g, [&](int64_t i) { return r[i]; });
    } else {
      pg = r[g] + beta * pold[g];
      qg = csys<T>(in, sc, p, g, [&](int64_t i) { return r[i] + beta * pold[i]; });
    }
    pnew[g] = pg;
    q[g] = qg;
    acc[0] += (double)pg * (double)qg;
  }
  block_sum<1>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    atomicAdd(&sc.acc_n[0], acc[0]);
    last = arrive_last(&sc.cnt_n, (uint32_t)in.nt_n);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    const double pq = ldv(&sc.acc_n[0]);
    sc.acc_n[0] = 0.0;
    if (pq > 0.0) {
      sc.alpha = sc.rr / pq;
    } else {
      sc.cg_active = 0;  // p^T C p <= 0: stop CG
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_upd(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                     InstScal *__restrict__ scal) {
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done || !sc.cg_active) return;
  const T *__restrict__ p = (const T *)(sc.pbuf ? in.p0 : in.p1);
  const T *__restrict__ q = (const T *)in.q;
  T *__restrict__ x = (T *)in.x;
  T *__restrict__ r = (T *)in.r;
  const T alpha = (T)sc.alpha;
  double acc[1] = {0.0};
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t g = tl.start + threadIdx.x + (int64_t)e * kThreads;
    if (g >= tl.start + tl.len) break;
    x[g] = x[g] + alpha * p[g];
    const T rv = r[g] - alpha * q[g];
    r[g] = rv;
    acc[0] += (double)rv * (double)rv;
  }
  block_sum<1>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    atomicAdd(&sc.acc_n[0], acc[0]);
    last = arrive_last(&sc.cnt_n, (uint32_t)in.nt_n);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    const double rr = ldv(&sc.acc_n[0]);
    sc.acc_n[0] = 0.0;
    sc.beta = rr / sc.rr;
    sc.rr = rr;
    sc.cg_steps += 1;
    sc.cg_total += 1;
    sc.pbuf ^= 1;
    bool more;
    if (in.cg_iters > 0) {
      more = sc.cg_steps < in.cg_iters;
    } else {  // Eq. cg_stop: ||r_j|| < 0.1 ||r_0||
      more = sc.cg_steps < in.cg_max && !(sqrt(rr) < 0.1 * sqrt(sc.rr0));
    }
    sc.cg_active = (more && rr > 0.0) ? 1 : 0;
  }
}

// --------------------------------------------------------------------------
// Set pass: relaxation, prox input, point-wise prox, dual update, stopping
// and adapt inner products (Algorithm PARSDMM FOR-body; Algorithm
// adapt-rho-gamma; Eqs. feas_stop, obj_stop)
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T clip(T w, double lo, double hi) {
  return fmin(fmax(w, (T)lo), (T)hi);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_setpass(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                      InstScal *__restrict__ scal, JobScal *__restrict__ jscal,
                                                      const JobDev *__restrict__ jobs) {
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  const int k = sc.k;
  const bool ad = adapt_iter(in, k);
  const bool ad_dots = ad && sc.have_k0;
  const bool chk = check_iter(in, k);
  const SegDev sg = in.seg[tl.item];
  const T *__restrict__ x = (const T *)in.x;
  // acc layout: 0..5 adapt dots, 6 feasD2 / ring, 7 s2, 8 s1, 9 wnorm
  double acc[kMaxHist + 2];
#pragma unroll
  for (int i = 0; i < kMaxHist + 2; ++i) acc[i] = 0.0;

  if (sg.kind == SEG_RING) {
    // x^k against the stored x^{k-1} .. x^{k-s} (Eq. obj_stop), then store x^k.
    T *__restrict__ ring = (T *)in.ring;
    const int H = in.hist;
    const int jmax = k < H ? k : H;
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
      const int64_t g = tl.start + threadIdx.x + (int64_t)e * kThreads;
      if (g >= tl.start + tl.len) break;
      const T xv = x[g];
      if (chk) {
        acc[0] += (double)xv * (double)xv;
        for (int j = 1; j <= jmax; ++j) {
          const int slot = (k - j) % H;
          const double d = (double)xv - (double)ring[(int64_t)slot * in.N + g];
          acc[j] += d * d;
        }
      }
      ring[(int64_t)(k % H) * in.N + g] = xv;
    }
    if (chk) {
      block_sum<kMaxHist + 1>(*reinterpret_cast<double(*)[kMaxHist + 1]>(acc));
      if (threadIdx.x == 0)
        for (int j = 0; j <= jmax; ++j) atomicAdd(&sc.acc_ring[j], acc[j]);
    }
  } else {
    const int b = sg.block;
    const BlockDev &bd = in.blk[b];
    const T rho = (T)sc.rho[b], irho = (T)sc.irho[b], gam = (T)sc.gamma[b];
    const T one_m_gam = (T)(1.0 - sc.gamma[b]);
    T *__restrict__ y = (T *)in.y;
    T *__restrict__ v = (T *)in.v;
    T *__restrict__ wbuf = (T *)in.w;
    T *__restrict__ sbuf = (T *)in.s;
    T *__restrict__ k0s = (T *)in.k0s;
    T *__restrict__ k0vh = (T *)in.k0vh;
    T *__restrict__ k0y = (T *)in.k0y;
    T *__restrict__ k0v = (T *)in.k0v;
    const T *__restrict__ m = (const T *)in.m;
    const int type = bd.type;
#pragma unroll
    for (int e = 0; e < kPerThread; ++e) {
      const int64_t row = tl.start + threadIdx.x + (int64_t)e * kThreads;
      if (row >= tl.start + tl.len) break;
      int64_t g;
      const T s = seg_forward<T>(in, sg.kind, x, row, g);
      const int64_t rb = sg.row0 + row;  // row inside the block
      const int64_t yi = bd.yoff + rb;
      const T y0 = y[yi], v0 = v[yi];
      const T xbar = gam * s + one_m_gam * y0;
      const T w = xbar - v0 * irho;
      if (ad) {
        // vhat^{k+1} = v^k + rho (y^k - s^{k+1}); dh = s - s^{k0}; dvh = vhat - vhat^{k0}
        const T vh = v0 + rho * (y0 - s);
        if (ad_dots) {
          const double dh = (double)s - (double)k0s[yi];
          const double dvh = (double)vh - (double)k0vh[yi];
          acc[0] += dh * dvh;
          acc[1] += dh * dh;
          acc[2] += dvh * dvh;
        }
        k0s[yi] = s;
        k0vh[yi] = vh;
      }
      if (type == BT_BOUNDS || type == BT_DIST) {
        T yn;
        if (type == BT_BOUNDS) {
          yn = clip<T>(w, bd.lo, bd.hi);
        } else {  // Eq. prox_sq_dist
          yn = (m[g] + rho * w) * (T)sc.inv1p[b];
        }
        const T vn = v0 + rho * (yn - xbar);
        y[yi] = yn;
        v[yi] = vn;
        if (ad) {
          if (ad_dots) {
            const double dg = -((double)yn - (double)k0y[yi]);
            const double dv = (double)vn - (double)k0v[yi];
            acc[3] += dg * dv;
            acc[4] += dg * dg;
            acc[5] += dv * dv;
          }
          k0y[yi] = yn;
          k0v[yi] = vn;
        }
        if (chk && type == BT_BOUNDS) {
          const double d = (double)s - (double)clip<T>(s, bd.lo, bd.hi);
          acc[6] += d * d;
          acc[7] += (double)s * (double)s;
        }
      } else {
        wbuf[bd.woff + rb] = w;
        if (type == BT_L2) acc[9] += (double)w * (double)w;
        if (type == BT_L1) acc[9] += fabs((double)w);
        if (chk) {
          acc[7] += (double)s * (double)s;
          if (type == BT_L1) acc[8] += fabs((double)s);
          if (type != BT_L2) sbuf[bd.soff + rb] = s;
        }
      }
    }
    block_sum<10>(*reinterpret_cast<double(*)[10]>(acc));
    if (threadIdx.x == 0) {
      double *a = sc.acc[b];
      if (ad_dots) {
        atomicAdd(&a[A_HV], acc[0]);
        atomicAdd(&a[A_HH], acc[1]);
        atomicAdd(&a[A_VHVH], acc[2]);
        if (type == BT_BOUNDS || type == BT_DIST) {
          atomicAdd(&a[A_GV], acc[3]);
          atomicAdd(&a[A_GG], acc[4]);
          atomicAdd(&a[A_VV], acc[5]);
        }
      }
      if (chk) {
        atomicAdd(&a[A_FEAS_D2], acc[6]);
        atomicAdd(&a[A_S2], acc[7]);
        atomicAdd(&a[A_S1], acc[8]);
      }
      if (type == BT_L1 || type == BT_L2) atomicAdd(&a[A_WNORM], acc[9]);
    }
  }

  // The last CTA of the instance resolves the l2 scales and arms the
  // selection jobs of this iteration.
  __shared__ bool last;
  if (threadIdx.x == 0) last = arrive_last(&sc.cnt_set, (uint32_t)in.nt_set);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  for (int b = 0; b < in.nb; ++b) {
    const BlockDev &bd = in.blk[b];
    const double *a = sc.acc[b];
    if (bd.type == BT_L2) {
      const double nrm = sqrt(ldv(&a[A_WNORM]));
      const double sg2 = sc.sigma[b];
      sc.l2scale[b] = nrm > sg2 ? sg2 / nrm : 1.0;
    }
    if (bd.job_w >= 0) {
      JobScal &js = jscal[bd.job_w];
      js.active = 1;
      js.pass = 0;
      js.prefix = 0;
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
  (void)jobs;
}

// --------------------------------------------------------------------------
// Radix selection (l1-ball threshold; top-k).  Keys are the bits of |value|,
// which order like the values.  Pass p histograms one 11-bit digit of the
// entries whose higher digits equal the prefix fixed so far; the last CTA of
// the job picks the bin holding the breakpoint and descends into it.
//   l1:  largest bin d with g(lo_d) >= tau, g(t) = sum_{|w|>t} (|w| - t):
//        the soft threshold theta lies at or above lo_d (Duchi et al.).
//   top-k: largest bin d with count(keys >= lo_d) >= k.
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_select(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                     InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                     JobScal *__restrict__ jscal, uint32_t *__restrict__ hcnt,
                                                     double *__restrict__ hs1, double *__restrict__ hs2, int pass) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  const Tile tl = tiles[blockIdx.x];
  const JobDev jd = jobs[tl.item];
  const InstDev &in = insts[jd.inst];
  InstScal &sc = scal[jd.inst];
  JobScal &js = jscal[tl.item];
  if (sc.done || !js.active || js.mode != JM_SELECT || js.pass != pass) return;

  extern __shared__ unsigned char smem_raw[];
  uint32_t *cnt = (uint32_t *)smem_raw;
  double *s1 = (double *)(smem_raw + kBins * sizeof(uint32_t));
  double *s2 = s1 + kBins;
  const bool need1 = jd.kind == JOB_L1;
  const bool need2 = jd.feas != 0;
  for (int i = threadIdx.x; i < kBins; i += kThreads) {
    cnt[i] = 0;
    s1[i] = 0.0;
    s2[i] = 0.0;
  }
  __syncthreads();

  const int hi = KT::kBits - pass * kDigitBits;
  const int lo = hi - kDigitBits > 0 ? hi - kDigitBits : 0;
  const K mask = (K)((1u << (hi - lo)) - 1u);
  const K pre = (K)js.prefix;
  const T *__restrict__ data = (const T *)(jd.feas ? in.s : in.w) + jd.data_off;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t row = tl.start + threadIdx.x + (int64_t)e * kThreads;
    const bool valid = row < tl.start + tl.len;
    int bin = -1;
    double a = 0.0;
    if (valid) {
      const T val = data[row];
      const K key = KT::key(val);
      if (hi >= KT::kBits || (key >> hi) == (pre >> hi)) {
        bin = (int)((key >> lo) & mask);
        a = fabs((double)val);
      }
    }
    // warp-aggregated histogram update: one shared atomic per distinct bin
    unsigned pending = __ballot_sync(0xffffffffu, bin >= 0);
    while (pending) {
      const int leader = __ffs(pending) - 1;
      const int lb = __shfl_sync(0xffffffffu, bin, leader);
      const unsigned grp = __ballot_sync(0xffffffffu, bin == lb);
      const bool mine = bin == lb;
      double v1 = (mine && need1) ? a : 0.0;
      double v2 = (mine && need2) ? a * a : 0.0;
      if (need1) v1 = warp_sum(v1);
      if (need2) v2 = warp_sum(v2);
      if (lane == leader) {
        atomicAdd(&cnt[lb], (uint32_t)__popc(grp));
        if (need1) atomicAdd(&s1[lb], v1);
        if (need2) atomicAdd(&s2[lb], v2);
      }
      pending &= ~grp;
    }
  }
  __syncthreads();
  uint32_t *gc = hcnt + jd.hist_off;
  double *g1 = hs1 + jd.hist_off;
  double *g2 = hs2 + jd.hist_off;
  for (int i = threadIdx.x; i < kBins; i += kThreads) {
    if (cnt[i]) {
      atomicAdd(&gc[i], cnt[i]);
      if (need1) atomicAdd(&g1[i], s1[i]);
      if (need2) atomicAdd(&g2[i], s2[i]);
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = arrive_last(&js.counter, (uint32_t)jd.ntiles);
  __syncthreads();
  if (!last) return;

  // ---- last CTA: choose the bin -------------------------------------------
  constexpr int kPer = kBins / kThreads;  // bins per thread
  const int nb = 1 << (hi - lo);
  // thread t owns bins [t*kPer, t*kPer + kPer)
  uint32_t c[kPer];
  double a1[kPer], a2[kPer];
  double tc = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int bi = threadIdx.x * kPer + j;
    c[j] = bi < nb ? *(volatile uint32_t *)&gc[bi] : 0u;
    a1[j] = (bi < nb && need1) ? ldv(&g1[bi]) : 0.0;
    a2[j] = (bi < nb && need2) ? ldv(&g2[bi]) : 0.0;
    tc += (double)c[j];
    t1 += a1[j];
    t2 += a2[j];
  }
  // exclusive suffix sums over threads (bins above this thread's range)
  __shared__ double suf[3][kThreads];
  suf[0][threadIdx.x] = tc;
  suf[1][threadIdx.x] = t1;
  suf[2][threadIdx.x] = t2;
  __syncthreads();
  // Hillis-Steele inclusive suffix scan
  for (int off = 1; off < kThreads; off <<= 1) {
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (threadIdx.x + off < kThreads) {
      v0 = suf[0][threadIdx.x + off];
      v1 = suf[1][threadIdx.x + off];
      v2 = suf[2][threadIdx.x + off];
    }
    __syncthreads();
    suf[0][threadIdx.x] += v0;
    suf[1][threadIdx.x] += v1;
    suf[2][threadIdx.x] += v2;
    __syncthreads();
  }
  double ac = js.c_above + suf[0][threadIdx.x] - tc;  // entries above my bins
  double as1 = js.s1_above + suf[1][threadIdx.x] - t1;
  double as2 = js.s2_above + suf[2][threadIdx.x] - t2;
  int best = -1;
  double bc = 0, b1 = 0, b2 = 0;  // "above" sums for the chosen bin
  for (int j = kPer - 1; j >= 0; --j) {
    const int bi = threadIdx.x * kPer + j;
    if (bi < nb) {
      const double cge = ac + (double)c[j];
      bool ok;
      if (jd.kind == JOB_L1) {
        const K lokey = pre | ((K)bi << lo);
        const double lov = KT::val(lokey);
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
    ac += (double)c[j];
    as1 += a1[j];
    as2 += a2[j];
  }
  // highest satisfying bin over the CTA
  __shared__ int sbest;
  if (threadIdx.x == 0) sbest = -1;
  __syncthreads();
  if (best >= 0) atomicMax(&sbest, best);
  __syncthreads();
  if (best >= 0 && best == sbest) {
    const int j = best - threadIdx.x * kPer;
    js.c_above = bc;
    js.s1_above = b1;
    js.s2_above = b2;
    const K np = pre | ((K)best << lo);
    js.prefix = (uint64_t)np;
    if (lo == 0) {  // final digit: the breakpoint key is exact
      if (jd.kind == JOB_L1) {
        js.theta = (b1 - js.tau) / bc;
      } else {
        js.need = js.k - (int64_t)bc;
        js.cK = (int64_t)c[j];
        js.kval = KT::val(np);
        js.tie_needed = (js.need < js.cK && np != 0) ? 1 : 0;
      }
    }
    js.pass = pass + 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += kThreads) {
    gc[i] = 0;
    g1[i] = 0.0;
    g2[i] = 0.0;
  }
}

// Tie counts per final-pass tile for card sets whose k-th value is tied.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ties(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                   InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                   JobScal *__restrict__ jscal, uint32_t *__restrict__ ties) {
  using KT = KeyOf<T>;
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  const BlockDev &bd = in.blk[tl.item];
  if (sc.done || bd.type != BT_CARD) return;
  const JobScal &js = jscal[bd.job_w];
  if (js.mode != JM_SELECT || !js.tie_needed) return;
  const typename KT::K K = (typename KT::K)js.prefix;
  const T *__restrict__ w = (const T *)in.w + bd.woff;
  int n = 0;
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t row = tl.start + threadIdx.x + (int64_t)e * kThreads;
    if (row < tl.start + tl.len && KT::key(w[row]) == K) ++n;
  }
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  if (n) atomicAdd(&tot, n);
  __syncthreads();
  if (threadIdx.x == 0) ties[jobs[bd.job_w].tie_off + tl.seq] = (uint32_t)tot;
}

// --------------------------------------------------------------------------
// Final pass: l1 / l2 / card prox from the stored w and the dual update
// v = v + rho (y - xbar) = rho (y - w), since w = xbar - v / rho.
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_final(const Tile *__restrict__ tiles, const InstDev *__restrict__ insts,
                                                    InstScal *__restrict__ scal, const JobDev *__restrict__ jobs,
                                                    const JobScal *__restrict__ jscal,
                                                    const uint32_t *__restrict__ ties) {
  using KT = KeyOf<T>;
  using K = typename KT::K;
  const Tile tl = tiles[blockIdx.x];
  const InstDev &in = insts[tl.inst];
  InstScal &sc = scal[tl.inst];
  if (sc.done) return;
  const int b = tl.item;
  const BlockDev &bd = in.blk[b];
  const int k = sc.k;
  const bool ad = adapt_iter(in, k);
  const bool ad_dots = ad && sc.have_k0;
  const T rho = (T)sc.rho[b];
  const T *__restrict__ w = (const T *)in.w + bd.woff;
  T *__restrict__ y = (T *)in.y + bd.yoff;
  T *__restrict__ v = (T *)in.v + bd.yoff;
  T *__restrict__ k0y = (T *)in.k0y + bd.yoff;
  T *__restrict__ k0v = (T *)in.k0v + bd.yoff;
  int mode = JM_ALL;
  double theta = 0.0;
  K K0 = 0;
  bool tie = false;
  int64_t need = 0, before = 0;
  if (bd.type != BT_L2) {
    const JobScal &js = jscal[bd.job_w];
    mode = js.mode;
    theta = js.theta;
    K0 = (K)js.prefix;
    tie = bd.type == BT_CARD && mode == JM_SELECT && js.tie_needed;
    need = js.need;
    if (tie) {  // ties in earlier tiles of this block
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
  const T scale = (T)sc.l2scale[b];
  const T th = (T)theta;
  double acc[3] = {0.0, 0.0, 0.0};
  __shared__ int wcount[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t row = tl.start + threadIdx.x + (int64_t)e * kThreads;
    const bool valid = row < tl.start + tl.len;
    const T wv = valid ? w[row] : T(0);
    T yn = T(0);
    if (bd.type == BT_L2) {
      yn = wv * scale;
    } else if (mode == JM_ALL) {
      yn = wv;
    } else if (mode == JM_NONE) {
      yn = T(0);
    } else if (bd.type == BT_L1) {
      const T a = fabs(wv) - th;
      yn = a > T(0) ? copysign(a, wv) : T(0);
    } else {
      // card: keep keys above the k-th key; at the k-th key keep all ties
      // unless the tie rule must choose (ranked below)
      const K key = KT::key(wv);
      yn = (key > K0 || (key == K0 && !tie)) ? wv : T(0);
    }
    if (tie) {
      // all threads take part in the ranked scan of this round
      const K key = KT::key(wv);
      const bool f = valid && key == K0;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) wcount[wid] = __popc(bal);
      __syncthreads();
      int pre = 0;
      for (int i = 0; i < wid; ++i) pre += wcount[i];
      int total = 0;
      for (int i = 0; i < kThreads / 32; ++i) total += wcount[i];
      const int rank = (int)before + pre + __popc(bal & ((1u << lane) - 1u));
      if (f) yn = rank < need ? wv : T(0);
      before += total;
      __syncthreads();
    }
    if (valid) {
      const T vn = rho * (yn - wv);
      y[row] = yn;
      v[row] = vn;
      if (ad) {
        if (ad_dots) {
          const double dg = -((double)yn - (double)k0y[row]);
          const double dv = (double)vn - (double)k0v[row];
          acc[0] += dg * dv;
          acc[1] += dg * dg;
          acc[2] += dv * dv;
        }
        k0y[row] = yn;
        k0v[row] = vn;
      }
    }
  }
  if (ad_dots) {
    block_sum<3>(acc);
    if (threadIdx.x == 0) {
      atomicAdd(&sc.acc[b][A_GV], acc[0]);
      atomicAdd(&sc.acc[b][A_GG], acc[1]);
      atomicAdd(&sc.acc[b][A_VV], acc[2]);
    }
  }
}

// --------------------------------------------------------------------------
// Per-instance tail: stopping quantities, Algorithm adapt-rho-gamma, C.
// --------------------------------------------------------------------------
__device__ void set_coefficients(const InstDev &in, InstScal &sc) {
  double c0 = in.alg1 ? 0.0 : 1.0, cz = 0.0, cx = 0.0, cy = 0.0;
  for (int b = 0; b < in.nb; ++b) {
    const double r = sc.rho[b];
    sc.irho[b] = 1.0 / r;
    sc.inv1p[b] = 1.0 / (1.0 + r);
    switch (in.blk[b].op) {
      case SIP_OP_I: c0 += r; break;
      case SIP_OP_DZ: cz += r; break;
      case SIP_OP_DX: cx += r; break;
      case SIP_OP_DY: cy += r; break;
      default: cz += r; cx += r; if (in.ndim == 3) cy += r; break;
    }
  }
  sc.c0 = c0;
  sc.cz = cz * in.ihz * in.ihz;
  sc.cx = cx * in.ihx * in.ihx;
  sc.cy = cy * in.ihy * in.ihy;
}

__device__ __forceinline__ double corr(double ab, double aa, double bb) {
  const double d = aa * bb;
  return d > 0.0 ? ab / sqrt(d) : 0.0;
}
__device__ __forceinline__ double spectral(double ab, double aa, double bb) {
  const double mg = ab / aa, sd = bb / ab;
  return 2.0 * mg > sd ? mg : sd - 0.5 * mg;
}

__global__ void k_tail(const InstDev *__restrict__ insts, InstScal *__restrict__ scal,
                       const JobScal *__restrict__ jscal, int ninst) {
  const int i = blockIdx.x;
  if (i >= ninst) return;
  const InstDev &in = insts[i];
  InstScal &sc = scal[i];
  if (sc.done) return;
  if (threadIdx.x == 0) {
    const int k = sc.k;
    const bool chk = check_iter(in, k);
    const bool ad = adapt_iter(in, k);
    double *tr = in.trace ? in.trace + (int64_t)(k - 1) * in.trace_w : nullptr;
    if (tr) {
      for (int b = 0; b < in.nb; ++b) {
        tr[b] = sc.rho[b];
        tr[in.nb + b] = sc.gamma[b];
      }
      tr[2 * in.nb] = sc.cg_steps;
      tr[2 * in.nb + 1] = __longlong_as_double(0x7ff8000000000000LL);
      for (int b = 0; b < in.p; ++b) tr[2 * in.nb + 2 + b] = __longlong_as_double(0x7ff8000000000000LL);
    }
    sc.iters = k;
    if (chk) {
      bool feas_ok = true;
      for (int b = 0; b < in.p; ++b) {
        const BlockDev &bd = in.blk[b];
        const double *a = sc.acc[b];
        const double s2 = a[A_S2];
        double d = 0.0;
        if (bd.type == BT_BOUNDS) {
          d = sqrt(a[A_FEAS_D2]);
        } else if (bd.type == BT_L2) {
          d = fmax(0.0, sqrt(s2) - sc.sigma[b]);
        } else {
          const JobScal &js = jscal[bd.job_s];
          if (js.mode == JM_ALL) {
            d = 0.0;
          } else if (js.mode == JM_NONE) {
            d = sqrt(s2);
          } else if (bd.type == BT_L1) {
            // s - P(s) = sign(s) min(|s|, theta)
            const double d2 = js.c_above * js.theta * js.theta + (s2 - js.s2_above);
            d = sqrt(fmax(d2, 0.0));
          } else {
            // card: ||s - P(s)||^2 = ||s||^2 - (squares of the k kept entries)
            const double d2 = s2 - js.s2_above - (double)js.need * js.kval * js.kval;
            d = sqrt(fmax(d2, 0.0));
          }
        }
        const double r = s2 > 0.0 ? d / sqrt(s2) : d;
        sc.r_feas[b] = r;
        if (!(r < in.eps_feas)) feas_ok = false;
        if (tr) tr[2 * in.nb + 2 + b] = r;
      }
      const int jmax = k < in.hist ? k : in.hist;
      double mx = 0.0;
      for (int j = 1; j <= jmax; ++j) mx = fmax(mx, sc.acc_ring[j]);
      const double xn = sqrt(sc.acc_ring[0]);
      sc.r_evol = xn > 0.0 ? sqrt(mx) / xn : sqrt(mx);
      if (tr) tr[2 * in.nb + 1] = sc.r_evol;
      if ((in.stop == 1 && feas_ok && sc.r_evol < in.eps_evol) || (in.stop == 2 && feas_ok)) {
        sc.done = 1;
        sc.stop_reason = 1;
      }
    }
    if (!sc.done) {
      if (ad) {
        if (sc.have_k0) {
          double nr[kMaxBlocks], ng[kMaxBlocks];
          for (int b = 0; b < in.nb; ++b) {
            const double *a = sc.acc[b];
            const double ac = corr(a[A_HV], a[A_HH], a[A_VHVH]);
            const double bc = corr(a[A_GV], a[A_GG], a[A_VV]);
            const bool aok = ac > in.eps_corr, bok = bc > in.eps_corr;
            const double ah = aok ? spectral(a[A_HV], a[A_HH], a[A_VHVH]) : 0.0;
            const double bh = bok ? spectral(a[A_GV], a[A_GG], a[A_VV]) : 0.0;
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
              r = sc.rho[b];
              g = 1.5;
            }
            if (in.adapt == 1) g = sc.gamma[b];
            nr[b] = r;
            ng[b] = fmin(g, in.gamma_max);
          }
          const double ref = in.alg1 ? nr[in.p] : 1.0;
          const double R = in.rho_ratio_max;
          for (int b = 0; b < in.p; ++b) nr[b] = fmin(fmax(nr[b], ref / R), ref * R);
          for (int b = 0; b < in.nb; ++b) {
            sc.rho[b] = nr[b];
            sc.gamma[b] = ng[b];
          }
        }
        sc.have_k0 = 1;
      }
      if (in.rho_sched && k < in.max_iter) {
        for (int b = 0; b < in.nb; ++b) {
          sc.rho[b] = in.rho_sched[(int64_t)k * in.nb + b];
          if (in.gamma_sched) sc.gamma[b] = in.gamma_sched[(int64_t)k * in.nb + b];
        }
      }
      set_coefficients(in, sc);
      sc.k = k + 1;
      if (k >= in.max_iter) sc.done = 1;
    }
  }
  __syncthreads();
  // clear the per-iteration accumulators
  double *acc = &sc.acc[0][0];
  for (int j = threadIdx.x; j < kMaxBlocks * kNAcc; j += blockDim.x) acc[j] = 0.0;
  for (int j = threadIdx.x; j <= kMaxHist; j += blockDim.x) sc.acc_ring[j] = 0.0;
}

}  // namespace sip

// ==========================================================================
// Per-call set-up: scalars, relative radii, non-finite model check.
// ==========================================================================
namespace sip {

__global__ void k_init(const InstDev *__restrict__ insts, InstScal *__restrict__ scal, int ninst) {
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
  sc.cg_active = 0;
  sc.cg_steps = 0;
  sc.cg_total = 0;
  sc.pbuf = 0;
  sc.have_k0 = 0;
  sc.nonfinite = 0;
  sc.cnt_n = sc.cnt_set = sc.cnt_norm = 0;
  sc.rr = sc.rr0 = sc.bnorm2 = sc.alpha = sc.beta = 0.0;
  sc.acc_n[0] = sc.acc_n[1] = 0.0;
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
#pragma unroll
  for (int e = 0; e < kPerThread; ++e) {
    const int64_t row = tl.start + threadIdx.x + (int64_t)e * kThreads;
    if (row >= tl.start + tl.len) break;
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
    if (bd.k_frac > 0.0) sc.kcard[b] = (int64_t)floor(bd.k_frac * (double)in.N);
    sc.acc[b][A_M1] = 0.0;
    sc.acc[b][A_M2] = 0.0;
  }
  if (*(volatile int *)&sc.nonfinite) {
    sc.done = 1;
    sc.stop_reason = -1;
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

cudaError_t launch_init(const Launch &L, const InstDev *insts, InstScal *scal, int ninst) {
  k_init<<<ninst, 32, 0, L.stream>>>(insts, scal, ninst);
  return cudaGetLastError();
}
cudaError_t launch_norms(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal) {
  SIP_DISPATCH(L, k_norms, nt, kThreads, 0, tiles, insts, scal);
  return cudaGetLastError();
}
cudaError_t launch_rhs(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal) {
  SIP_DISPATCH(L, k_rhs, nt, kThreads, 0, tiles, insts, scal);
  return cudaGetLastError();
}
cudaError_t launch_cg_dir(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal) {
  SIP_DISPATCH(L, k_cg_dir, nt, kThreads, 0, tiles, insts, scal);
  return cudaGetLastError();
}
cudaError_t launch_cg_upd(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal) {
  SIP_DISPATCH(L, k_cg_upd, nt, kThreads, 0, tiles, insts, scal);
  return cudaGetLastError();
}
cudaError_t launch_setpass(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                           JobScal *jscal, const JobDev *jobs) {
  SIP_DISPATCH(L, k_setpass, nt, kThreads, 0, tiles, insts, scal, jscal, jobs);
  return cudaGetLastError();
}
static constexpr size_t kSelectSmem = kBins * (sizeof(uint32_t) + 2 * sizeof(double));
cudaError_t launch_select(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                          const JobDev *jobs, JobScal *jscal, uint32_t *hcnt, double *hs1, double *hs2, int pass) {
  // 40 KB of dynamic shared memory: below the 48 KB default, no opt-in needed
  static_assert(kSelectSmem <= 48 * 1024, "select histogram exceeds the default shared-memory limit");
  SIP_DISPATCH(L, k_select, nt, kThreads, kSelectSmem, tiles, insts, scal, jobs, jscal, hcnt, hs1, hs2, pass);
  return cudaGetLastError();
}
int select_passes(int dtype) { return dtype == SIP_F64 ? num_passes<double>() : num_passes<float>(); }
cudaError_t launch_ties(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                        const JobDev *jobs, JobScal *jscal, uint32_t *ties) {
  SIP_DISPATCH(L, k_ties, nt, kThreads, 0, tiles, insts, scal, jobs, jscal, ties);
  return cudaGetLastError();
}
cudaError_t launch_final(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const JobDev *jobs, const JobScal *jscal, const uint32_t *ties) {
  SIP_DISPATCH(L, k_final, nt, kThreads, 0, tiles, insts, scal, jobs, jscal, ties);
  return cudaGetLastError();
}
cudaError_t launch_tail(const Launch &L, const InstDev *insts, InstScal *scal, const JobScal *jscal, int ninst) {
  k_tail<<<ninst, 32, 0, L.stream>>>(insts, scal, jscal, ninst);
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
