// Device-side data model of the PARSDMM engine (internal to libsip.so).
//
// One "instance" is one projection problem (grid, blocks, state arena).  A
// plan holds one or many instances of one dtype; every kernel walks a tile
// list in which each tile names its instance, so one launch serves a single
// large grid or a ragged batch of small ones alike.
//
// Blocks follow the paper's stacked variables (Eq. conc_variables): blocks
// 0..p-1 are the user's sets (A_i, C_i); in the paper's form block p is the
// identity block A_{p+1} = I_N with the prox of the squared distance
// (Eq. prox_sq_dist).  A block's rows y_i, v_i are contiguous in the
// instance's y / v arrays at offset yoff.  A block whose operator is the TV
// stack has one segment per difference operator; every other block has one
// segment.  Segment rows decompose on the operator's own output grid, z
// fastest (Eq. FD_mat).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sip.h"

namespace sip {

constexpr int kMaxSets = SIP_MAX_SETS;
constexpr int kMaxBlocks = kMaxSets + 1;
constexpr int kMaxSegs = kMaxBlocks * 3 + 1;
constexpr int kMaxHist = 8;          // s of Eq. obj_stop, upper limit
constexpr int kThreads = 256;        // threads per CTA for the streaming kernels
constexpr int kPerThread = 4;
constexpr int kTile = kThreads * kPerThread;
// Grid-point work items of an instance with a blur block: blocks of kBlurTZ
// z rows times kBlurTA samples along the blur axis (x or y), or for a blur
// along z runs of at most kBlurLen samples of one z column; staged in
// shared memory with the kernel's halo of up to 2 SIP_MAX_BLUR_RADIUS
// samples along the axis.
constexpr int kBlurTZ = 32;
constexpr int kBlurTA = 32;
constexpr int kBlurLen = 1024;
constexpr int kBlurBuf = (kBlurTZ + 2) * (kBlurTA + 4 * SIP_MAX_BLUR_RADIUS);  // rows z0-1 .. z0+kBlurTZ
static_assert(kBlurTZ * kBlurTA <= kBlurLen && kBlurLen + 4 * SIP_MAX_BLUR_RADIUS <= kBlurBuf,
              "a staged block fits the buffer");
constexpr int64_t kMaxChunk = 64 * kTile;  // rows of one work item, at most
constexpr int kDigitBits = 11;       // radix digit of the selection passes
constexpr int kBins = 1 << kDigitBits;

enum SegKind : int32_t { SEG_I = 0, SEG_DZ = 1, SEG_DX = 2, SEG_DY = 3, SEG_RING = 4, SEG_BLUR = 5 };
// BT_ANNULUS: the annulus on A x as a whole; BT_LINE: a set applied to
// every line of A x on its own (BlockDev.line_type says which).
enum BlkType : int32_t { BT_BOUNDS = 0, BT_L1 = 1, BT_L2 = 2, BT_CARD = 3, BT_DIST = 4, BT_ANNULUS = 5, BT_LINE = 6 };
enum JobKind : int32_t { JOB_L1 = 0, JOB_TOPK = 1 };
// How a selection job resolved: run the radix select, or the set keeps
// everything (inside the ball / k >= M), or nothing (tau = 0 / k = 0).
enum JobMode : int32_t { JM_SELECT = 0, JM_ALL = 1, JM_NONE = 2 };

// Per-block binary64 accumulators (one iteration).
enum Acc : int32_t {
  A_WNORM = 0,   // ||w||_2^2 (l2 set) or ||w||_1 (l1 set)
  A_FEAS_D2,     // ||s - P(s)||^2 for bounds sets
  A_S2,          // ||s||^2
  A_S1,          // ||s||_1
  A_HV, A_HH, A_VHVH,   // adapt-rho-gamma: dh.dvh, dh.dh, dvh.dvh
  A_GV, A_GG, A_VV,     // adapt-rho-gamma: dg.dv, dg.dg, dv.dv
  A_M1, A_M2,    // ||A m||_1, ||A m||_2^2 (relative radii)
  kNAcc
};

// Division by a fixed divisor d >= 1 for 0 <= n < 2^31 by a multiply-high
// and a shift (Granlund and Montgomery's round-up method):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (mulhi(n, m) + n) >> l.
struct FastDiv {
  uint32_t d, m, s;
};

#ifdef __CUDACC__
__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(n, f.m);
#else
  const uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (uint32_t)(((uint64_t)t + n) >> f.s);
}
#endif

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  if (d == 0) d = 1;
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  f.d = d;
  f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  f.s = l;
  return f;
}

struct Tile {
  int32_t inst;   // instance
  int32_t item;   // segment (set pass), block (final pass) or job (select)
  int64_t start;  // first row / grid point
  int32_t len;    // rows in this work item (a CTA walks it kTile rows at a time)
  int32_t seq;    // tile number inside its item (tie ranks)
};

struct SegDev {
  int32_t kind;   // SegKind
  int32_t block;  // owning block (-1 for the x-history ring)
  int64_t row0;   // first row of the segment inside its block
  int64_t len;    // rows
};

struct BlockDev {
  int32_t op, type;      // sip_op, BlkType
  int64_t M;             // rows of A_i
  int64_t yoff;          // offset into y, v and the adapt copies
  int64_t woff;          // offset into the w scratch (l1/l2/card), -1 otherwise
  int64_t soff;          // offset into the s scratch (l1/card feasibility), -1
  double lo, hi;         // bounds
  double sigma_abs, sigma_rel, k_frac;
  int64_t k_abs;
  int32_t job_w, job_s;  // selection jobs (global index) or -1
  int32_t seg0, nseg;
  // BT_LINE: the simple set of every line (BT_L1, BT_L2, BT_CARD or
  // BT_ANNULUS) and the lines on the operator's output grid (z fastest):
  // line j holds line_len entries line_stride apart from
  // (j % line_a) + (j / line_a) * line_b, with (line_a, line_b) = (1, len)
  // along z, (n_z', n_z' n_x') along x and (n_z' n_x', 0) along y
  int32_t line_type, scope;
  int64_t line_len, line_stride, nlines, line_a, line_b;
  // per-entry bounds (point-wise data fit): lo at bv_lo, hi at bv_hi of the
  // instance's bvec array, M entries each; -1: the scalar lo / hi apply
  int64_t bv_lo, bv_hi;
};

struct JobDev {
  int32_t inst, block, kind, feas;  // feas: selection on s = A x (Eq. feas_stop)
  int64_t M;
  int64_t data_off;   // into w or s scratch
  int64_t hist_off;   // into the histogram arrays (kBins per job)
  int64_t tie_off;    // into the tie-count array (one per tile)
  int32_t ntiles;
  int32_t pad;
  void *cand;         // card w-jobs: kWinCap window candidates (keys), else null
};

// Window candidates per cardinality job (keys of |w| inside the window),
// and the window's half-width relative to the last k-th value: initial,
// smallest and largest.
constexpr int kWinCap = 4096;
constexpr double kWinRel0 = 1.0 / 32, kWinRelMin = 1.0 / 4096, kWinRelMax = 0.5;

struct JobScal {
  int32_t active, mode, pass, tie_needed;
  uint32_t counter;
  int32_t pad;
  uint64_t prefix;    // fixed high key bits so far; final key after the last pass
  uint64_t n_above;   // entries with key above the current bin (count)
  double c_above, s1_above, s2_above;  // the same count; sums of |w| and w^2 over them
  double tau;         // l1 radius
  int64_t k;          // cardinality
  double theta;       // l1 soft threshold
  int64_t need;       // card: ties to keep at the final key
  int64_t cK;         // card: entries equal to the final key
  double kval;        // card: |value| of the final key
  float thetaf;       // theta in binary32
  int32_t pad2;
  // Warm-started window of the top-k selection (card w-jobs).  The set pass
  // counts the entries with |w| above win_hi and stores the keys inside
  // [win_lo, win_hi] (bounds rounded to the storage type); when the k-th key
  // falls inside, one CTA selects it from the candidates and the radix
  // passes are skipped.  The tail re-centres the window on each iteration's
  // k-th value.
  double win_lo, win_hi;   // window bounds on |w|
  double win_rel;          // half-width relative to the last k-th value
  uint64_t win_above;      // entries above the window (this iteration)
  uint32_t win_n;          // entries inside the window (may exceed kWinCap)
  int32_t win_on;          // the set pass collects
  int32_t win_hit;         // this iteration's selection came from the window
  int32_t pad3;
};

struct InstDev {
  int32_t nz, nx, ny, ndim;
  FastDiv fz, fx, fzm, fxm;  // division by n_z, n_x, n_z - 1, n_x - 1
  double ihz, ihx, ihy;      // 1/h per axis
  float ihzf, ihxf, ihyf;    // the same in binary32
  int32_t pad0;
  int64_t N;
  int32_t nb, p, alg1, nseg, njob, job0;
  int32_t nt_n, nt_set, nt_fin;
  // this instance's first work item in each plan-wide list (lists hold the
  // instances' items one instance after another), and its selection and
  // per-line item counts
  int32_t tn0, tset0, tsel0, tfin0, tline0, nt_sel, nt_line, pad_t;
  int32_t nt_rhs;            // work items of the staged right-hand side list (0: none)
  int32_t nt_part;           // per-tile partial sums per quantity: max(nt_n, nt_rhs)
  int32_t hist;              // evol_hist
  // options
  int32_t max_iter, cg_iters, cg_max, check_every, stop, adapt, adapt_every;
  double eps_feas, eps_evol, rho0, gamma0, eps_corr, rho_ratio_max, gamma_max;
  const double *rho_sched, *gamma_sched;  // device copies, may be null
  double *trace;             // device trace rows, may be null
  uint32_t *ndone;           // plan-wide count of finished instances
  uint32_t *err;             // plan-wide device error word (a bounded wait that ran out)
  int32_t trace_w;
  int32_t select_window;     // option: warm-started window for top-k selections
  int32_t k0_ring;           // s^{k0} from x^{k0} in the history ring (adapt_every < hist), no k0s copy
  int32_t bf16;              // option: y_i, v_i (and their adapt copies) rounded to bfloat16 at every store
  // blurring forward operator F of a data-fit block (bl_R = 0: none):
  // radius, axis (0 z, 1 x, 2 y), samples along the axis, the block, the
  // stride of one step along the axis, and the blur table in the storage
  // type (in bvec at bl_off): the taps k_0..k_R, the autocorrelation
  // a_0..a_2R of the kernel (F^T F away from the ends) and the R x R
  // correction E[i][l] = sum_{j<0} k_|i-j| k_|l-j| of the first R samples
  int32_t bl_R, bl_axis, bl_n, bl_blk;
  int32_t bl_box;  // every tap equal (a box, e.g. a motion blur): window sums slide along the axis
  int32_t bl_pad;
  int64_t bl_st, bl_off;
  const void *bl_w;
  void *bl_s;  // s = F x of the current iteration (N entries), read by the set pass
  // device arrays, element type = the plan's dtype
  const void *m;
  void *x, *ring, *y, *v, *w, *s, *k0s, *k0vh, *k0y, *k0v;
  void *bvec;  // per-entry bound vectors of the blocks that have them
  // conjugate-gradient vectors: residual r, w = C r and s = C p are double
  // buffered (read at stencil neighbours while the next values are written);
  // the direction p is updated in place
  void *cr[2], *cw[2], *cs[2], *cp;
  // per-tile partial sums of the grid-point launches, in the accumulator
  // type (binary32 for binary32 storage): 3 slots x 2 quantities x nt_n,
  // slot 0 r.r of the right-hand side launch, slots 1 and 2 alternate
  // between the CG launches
  void *cgp;
  BlockDev blk[kMaxBlocks];
  SegDev seg[kMaxSegs];
};

// The fields of an instance the CG launches read, passed by value to the
// launches of single-instance plans (same names as in InstDev).
struct CgDesc {
  int32_t nz, nx, ny, cg_iters, cg_max, nt_part;
  FastDiv fz, fx;
  int64_t N;
  uint32_t *err;  // the plan's device error word (index guards of debug builds)
  void *x, *cp, *cgp;
  void *cr[2], *cw[2], *cs[2];
  int32_t bl_R, bl_axis, bl_n, bl_blk;
  int64_t bl_st;
  const void *bl_w;
};
struct CgOne {
  CgDesc d;
  int64_t chunk;  // points per grid-point work item
  int32_t on;     // single-instance plan: work item b = points [b chunk, (b+1) chunk)
  int32_t pad;
};
inline CgDesc cg_desc(const InstDev &in) {
  CgDesc d;
  d.nz = in.nz;
  d.nx = in.nx;
  d.ny = in.ny;
  d.cg_iters = in.cg_iters;
  d.cg_max = in.cg_max;
  d.nt_part = in.nt_part;
  d.fz = in.fz;
  d.fx = in.fx;
  d.N = in.N;
  d.err = in.err;
  d.x = in.x;
  d.cp = in.cp;
  d.cgp = in.cgp;
  for (int j = 0; j < 2; ++j) {
    d.cr[j] = in.cr[j];
    d.cw[j] = in.cw[j];
    d.cs[j] = in.cs[j];
  }
  d.bl_R = in.bl_R;
  d.bl_axis = in.bl_axis;
  d.bl_n = in.bl_n;
  d.bl_blk = in.bl_blk;
  d.bl_st = in.bl_st;
  d.bl_w = in.bl_w;
  return d;
}

// A single-instance plan's descriptor as a launch parameter (on = 1):
// kernels then address their arrays without reading the descriptor from
// memory first.  Valid while the descriptor does not change after the
// plan is built (the plan owns its model copy).
struct InstOne {
  InstDev d;
  int32_t on;
  int32_t pad;
};

// Conjugate-gradient state between step launches.  Every CTA of a step
// launch derives it from the previous launch's partial sums and the previous
// state; the instance's first tile stores it in slot (phase & 1) while the
// launch reads slot ((phase - 1) & 1).
struct CgState {
  double alpha, rr, rr0;  // step length; r.r; r_0.r_0 (binary64 storage)
  float alphaf, rrf, rr0f;  // the same for binary32 storage
  int32_t active, steps;  // this launch takes a step; steps taken before it
};

struct InstScal {
  int32_t k;            // iteration in progress (1-based)
  int32_t done;         // stopping rule held (or a non-finite model); kernels no-op
  int32_t iters, stop_reason;
  int32_t cg_steps, cg_total;  // CG steps of the last iteration; of the run
  int32_t have_k0, nonfinite;
  uint32_t cnt_set, cnt_norm;
  int32_t win_hits;     // top-k selections resolved from their window (run total)
  int32_t pad_w;
  CgState cg[2];
  double rho[kMaxBlocks], gamma[kMaxBlocks], irho[kMaxBlocks], inv1p[kMaxBlocks];
  double l2scale[kMaxBlocks];
  double c0, cz, cx, cy;
  // binary32 copies written next to the binary64 values, so binary32
  // kernels convert nothing: c0, cz, cx, cy and per block
  // rho, 1/rho, gamma, 1-gamma, 1/(1+rho), l2 scale
  float cf[4];
  float bf[kMaxBlocks][6];
  double sigma[kMaxBlocks];
  int64_t kcard[kMaxBlocks];
  double r_feas[kMaxSets];
  double r_evol;
  double acc[kMaxBlocks][kNAcc];
  double acc_ring[kMaxHist + 1];
};

// Type traits for the radix keys of |value|.
template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
  using K = uint32_t;
  static constexpr int kBits = 31;  // sign bit of |v| is zero
  static __device__ __forceinline__ K key(float v) { return __float_as_uint(fabsf(v)); }
  static __device__ __forceinline__ double val(K k) { return (double)__uint_as_float((uint32_t)k); }
};
template <> struct KeyOf<double> {
  using K = uint64_t;
  static constexpr int kBits = 63;
  static __device__ __forceinline__ K key(double v) { return (K)__double_as_longlong(fabs(v)); }
  static __device__ __forceinline__ double val(K k) { return __longlong_as_double((long long)k); }
};

template <typename T> constexpr int num_passes() { return (KeyOf<T>::kBits + kDigitBits - 1) / kDigitBits; }

// Index guards of debug builds (compiled with -DSIP_GUARDS, the library
// libsip_guarded.so): a work item or an index outside its array records
// SIP_ERR_INTERNAL in the plan's error word (err[0]), the number of the
// check (err[1]) and the offending index (err[3], err[4]: low and high
// words), and the access is skipped; the host reports it after the
// projection.  Release builds compile the guards away.
#if defined(__CUDACC__) && defined(SIP_GUARDS)
static __device__ __noinline__ void guard_fail(uint32_t *err, uint32_t check, int64_t idx) {
  if (err && atomicCAS(err, 0u, (uint32_t)SIP_ERR_INTERNAL) == 0u) {
    err[1] = check;
    err[3] = (uint32_t)((uint64_t)idx & 0xffffffffu);
    err[4] = (uint32_t)((uint64_t)idx >> 32);
    __threadfence();
  }
}
// a CTA-uniform check at a work item's start: the whole CTA leaves the item
#define SIP_GUARD_TILE(ERR, OK, CHECK, IDX)                                  \
  do {                                                                       \
    if (!(OK)) {                                                             \
      if (threadIdx.x == 0) ::sip::guard_fail((ERR), (CHECK), (int64_t)(IDX)); \
      return;                                                                \
    }                                                                        \
  } while (0)
// a per-thread check of one index: false (after recording) when it fails
#define SIP_GUARD_IDX(ERR, OK, CHECK, IDX) \
  ((OK) ? true : (::sip::guard_fail((ERR), (CHECK), (int64_t)(IDX)), false))
#else
#define SIP_GUARD_TILE(ERR, OK, CHECK, IDX) \
  do {                                      \
  } while (0)
#define SIP_GUARD_IDX(ERR, OK, CHECK, IDX) true
#endif

}  // namespace sip
