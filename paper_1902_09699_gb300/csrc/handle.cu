// extern "C" entry points of libsip.so (declared in include/sip.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sip.h"
#include "sip_dev.cuh"
#include "sip_host.h"
#include "sip_kernels.h"

using namespace sip;

struct sip_handle {
  Plan lev[SIP_MAX_LEVELS];  // lev[0]: finest grid; lev[l]: the grid coarsened l times (ML-PARSDMM)
  int levels = 1;
  int batch = 0;    // > 0: a batched handle of `batch` instances (packed buffers)
  bool dykstra = false;  // parallel Dykstra: the batch holds the p single-set sub-problems
  void *dk_x = nullptr;  // its iterate x
  sip_options opts;
  sip_grid grid;
  std::vector<sip_set> sets;
  cudaStream_t cap = nullptr;  // private stream used only to capture graphs
  int32_t *pinned = nullptr;   // pinned flag for the stopping-rule poll
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timing = false;
  bool warm_next = false;  // sip_set_state loaded x, y, v: the next projection starts from them
  bool warm_pen = false;   // ... and starting rho_i, gamma_i (warm_rho, warm_gamma)
  std::vector<double> warm_rho, warm_gamma;
  KernelTimer timer;
  std::string err;
  // the instances as built (before plan_build resolves them), for rebuilding
  // the plan with other launch-shape knobs; single-level and batched handles
  std::vector<InstLayout> layouts0;
  // adapt-rho-gamma's saved quantities for the next warm start (v-hat, y, v
  // at k0 and x^{k0}), staged until the projection's preparation
  void *k0_stage = nullptr;
  bool warm_k0 = false;
  bool tuned = false;     // the first projection's tuning has run (or was not asked for)
  sip_tuning report;      // what tuning measured
};

namespace {

#define CKH(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(SIP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t esz(int dtype) { return dtype == SIP_F64 ? 8 : 4; }

sip_status keep(sip_handle *h, sip_status s) {
  if (h && s != SIP_OK) h->err = g_err;
  return s;
}

// The plan's device error word after a projection (control words [2], [3],
// [5], [6]): a bounded wait that ran out, or, in builds with index guards,
// the first guard that failed and its index.
sip_status device_error(const uint32_t ctrl[8]) {
  if (ctrl[2] == (uint32_t)SIP_ERR_INTERNAL)
    return fail(SIP_ERR_INTERNAL, "device index guard %u failed at index %lld", ctrl[3],
                (long long)(((uint64_t)ctrl[6] << 32) | ctrl[5]));
  return fail(SIP_ERR_TIMEOUT, "a bounded device wait ran out (a grid barrier or a bulk copy did not complete)");
}

sip_grid coarse_of(const sip_grid &g) {
  sip_grid c = g;
  for (int a = 0; a < g.ndim; ++a) {
    c.n[a] = (g.n[a] + 1) / 2;
    c.h[a] = 2.0 * g.h[a];
  }
  return c;
}

// minimal InstDev describing one grid and the parts of one operator
InstDev op_inst(const GridDesc &g, int op) {
  InstDev d;
  memset(&d, 0, sizeof d);
  d.nz = (int32_t)g.n[0];
  d.nx = (int32_t)g.n[1];
  d.ny = (int32_t)g.n[2];
  d.ndim = g.ndim;
  set_fastdiv(d);
  d.ihz = 1.0 / g.h[0];
  d.ihx = 1.0 / g.h[1];
  d.ihy = 1.0 / g.h[2];
  d.ihzf = (float)d.ihz;
  d.ihxf = (float)d.ihx;
  d.ihyf = (float)d.ihy;
  d.N = g.N();
  int64_t row0 = 0;
  for (int kind : op_parts(g, op)) {
    SegDev &s = d.seg[d.nseg++];
    s.kind = kind;
    s.block = 0;
    s.row0 = row0;
    s.len = part_rows(g, kind);
    row0 += s.len;
  }
  return d;
}

// Temporary device copy of a small host struct (single-step calls only).
template <typename S>
struct DevCopy {
  S *p = nullptr;
  cudaError_t make(const S &h) {
    cudaError_t e = cudaMalloc(&p, sizeof(S));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(p, &h, sizeof(S), cudaMemcpyHostToDevice);
  }
  ~DevCopy() {
    if (p) cudaFree(p);
  }
};

sip_status check_grid_op(const sip_grid *grid, int op) {
  if (!grid) return fail(SIP_ERR_INVALID_ARG, "grid is NULL");
  sip_set s;
  memset(&s, 0, sizeof s);
  s.op = op;
  s.type = SIP_SET_BOUNDS;
  s.lo = -INFINITY;
  s.hi = INFINITY;
  sip_options o;
  sip_options_default(&o);
  return validate(grid, &s, 1, &o);
}

}  // namespace

extern "C" {

void sip_options_default(sip_options *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->max_iter = 200;
  o->cg_iters = 5;
  o->cg_max = 100;
  o->eps_feas = 1e-3;
  o->eps_evol = 1e-2;
  o->check_every = 5;
  o->evol_hist = 5;
  o->stop = 0;
  o->adapt = 1;
  o->adapt_every = 2;
  o->rho0 = 1.0;
  o->gamma0 = 1.5;
  o->eps_corr = 0.3;
  o->rho_ratio_max = 1e3;
  o->gamma_max = 1.99;
  o->form = SIP_FORM_ALG1;
  o->dtype = SIP_F32;
  o->levels = 1;
  o->coarse_iter = 0;
  o->select_window = 1;
  o->cluster_ctas = 0;
  o->tune = 0;
  o->store_bf16 = 0;
}

const char *sip_last_error(const sip_handle *h) {
  if (h && !h->err.empty()) return h->err.c_str();
  return g_err.c_str();
}

sip_status sip_create(const sip_grid *grid, const sip_set *sets, int nsets, const sip_options *opts,
                      sip_handle **out) {
  if (!out) return fail(SIP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sip_status st = validate(grid, sets, nsets, opts);
  if (st) return st;
  sip_grid grids[SIP_MAX_LEVELS];
  grids[0] = *grid;
  for (int l = 1; l < opts->levels; ++l) {
    grids[l] = coarse_of(grids[l - 1]);
    if ((st = validate(&grids[l], sets, nsets, opts))) return fail(st, "level %d: %s", l, g_err.c_str());
  }
  sip_handle *h = new (std::nothrow) sip_handle();
  if (!h) return fail(SIP_ERR_OOM, "host allocation failed");
  h->opts = *opts;
  h->grid = *grid;
  h->sets.assign(sets, sets + nsets);
  h->levels = opts->levels;
  auto bail = [&](sip_status s) {
    sip_destroy(h);
    return s;
  };
  {
    std::vector<InstLayout> L{make_layout(grid_desc(*grid), sets, nsets, *opts)};
    if (opts->levels == 1) h->layouts0 = L;
    if ((st = plan_build(h->lev[0], L, opts->dtype, true))) return bail(st);
  }
  memset(&h->report, 0, sizeof h->report);
  for (int l = 1; l < opts->levels; ++l) {
    sip_options oc = *opts;
    oc.max_iter = opts->coarse_iter > 0 ? opts->coarse_iter : opts->max_iter;
    std::vector<InstLayout> L{make_layout(grid_desc(grids[l]), sets, nsets, oc)};
    if ((st = plan_build(h->lev[l], L, opts->dtype, true))) return bail(st);
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&h->pinned, sizeof(int32_t)) != cudaSuccess || cudaEventCreate(&h->ev0) != cudaSuccess ||
      cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(SIP_ERR_CUDA, "stream/event set-up failed"));
  }
  *out = h;
  return SIP_OK;
}

sip_status sip_destroy(sip_handle *h) {
  if (!h) return SIP_OK;
  if (h->dk_x) cudaFree(h->dk_x);
  if (h->k0_stage) cudaFree(h->k0_stage);
  for (auto &P : h->lev) P.release();
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
  return SIP_OK;
}

int64_t sip_device_bytes(const sip_handle *h) {
  if (!h) return 0;
  int64_t b = 0;
  for (const auto &P : h->lev) b += P.arena_bytes;
  return b;
}

double sip_bytes_per_iter(const sip_handle *h) {
  if (!h || h->lev[0].layouts.empty()) return 0.0;
  double b = 0.0;
  for (const auto &L : h->lev[0].layouts) b += layout_bytes_per_iter(L, h->opts.dtype);
  return b;
}

static sip_status prolong_state(Plan &C, Plan &F, cudaStream_t st) {
  const Launch L{F.dtype, st};
  const InstLayout &lc = C.layouts[0], &lf = F.layouts[0];
  const InstDev &dc = C.h_insts[0], &df = F.h_insts[0];
  const size_t W = esz(F.dtype);
  int64_t cd[3], fd[3];
  int stag;
  part_dims(lc.g, SEG_I, cd, stag);
  part_dims(lf.g, SEG_I, fd, stag);
  CKH(launch_prolong(L, cd, fd, -1, dc.x, df.x));
  for (int b = 0; b < dc.nb; ++b) {
    const BlockDev &bc = dc.blk[b], &bf = df.blk[b];
    for (int s = 0; s < bc.nseg; ++s) {
      const SegDev &sc = dc.seg[bc.seg0 + s], &sf = df.seg[bf.seg0 + s];
      part_dims(lc.g, sc.kind, cd, stag);
      part_dims(lf.g, sf.kind, fd, stag);
      const int64_t oc = (bc.yoff + sc.row0) * W, of = (bf.yoff + sf.row0) * W;
      CKH(launch_prolong(L, cd, fd, stag, (char *)dc.y + oc, (char *)df.y + of));
      CKH(launch_prolong(L, cd, fd, stag, (char *)dc.v + oc, (char *)df.v + of));
    }
  }
  return SIP_OK;
}

// Starting rho_i, gamma_i of a warm start, written over the rho0 / gamma0
// values of the initialisation in stream order, before the first iteration;
// the scalars derived from them come from the device's own coefficient
// update (launch_load_penalties).
static sip_status load_penalties(sip_handle *h, Plan &F, cudaStream_t st) {
  const InstDev &in = F.h_insts[0];
  Penalties pen;
  memset(&pen, 0, sizeof pen);
  for (int b = 0; b < in.nb; ++b) {
    pen.rho[b] = h->warm_rho[b];
    pen.gamma[b] = h->warm_gamma[b];
  }
  CKH(launch_load_penalties(st, F.d_insts, F.d_scal, pen));
  return SIP_OK;
}

// The staged adapt-rho-gamma quantities into place after the preparation
// (which clears them): the copies at k0, x^{k0} in the history-ring slot the
// first adapt call reads, and the flag that makes that call form its
// differences.
static sip_status load_adapt_state(sip_handle *h, Plan &F, cudaStream_t st) {
  const InstDev &d = F.h_insts[0];
  const size_t W = esz(h->opts.dtype), M = (size_t)F.layouts[0].Mtot, N = (size_t)d.N;
  const char *src = (const char *)h->k0_stage;
  const int H = d.hist, ae = d.adapt_every;
  const int slot = ((1 - ae) % H + H) % H;
  CKH(cudaMemcpyAsync(d.k0vh, src, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync(d.k0y, src + M * W, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync(d.k0v, src + 2 * M * W, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync((char *)d.ring + (size_t)slot * N * W, src + 3 * M * W, N * W, cudaMemcpyDeviceToDevice, st));
  static const int32_t one = 1;
  CKH(cudaMemcpyAsync(&F.d_scal->have_k0, &one, sizeof one, cudaMemcpyHostToDevice, st));
  return SIP_OK;
}

// ----------------------------------------------------------------------------
// plan tuning (sip_tuning): coordinate search over launch-shape knobs,
// measured on the handle's own model, cached process-wide per shape
// ----------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, sip_tuning> g_tune_cache;

static bool tunable(const sip_handle *h) { return !h->layouts0.empty() && !h->dykstra && h->levels == 1; }

// Everything the knobs' effect depends on: dtype, options, every instance's
// grid and blocks.
static std::string tune_key(const sip_handle *h) {
  char buf[160];
  const sip_options &o = h->opts;
  snprintf(buf, sizeof buf, "t%d b%d f%d cg%d/%d a%d/%d w%d e%d c%d s%d;", o.dtype, h->batch, o.form, o.cg_iters,
           o.cg_max, o.adapt, o.adapt_every, o.select_window, o.exec, o.cluster_ctas, o.stop);
  std::string k = buf;
  for (const InstLayout &L : h->layouts0) {
    snprintf(buf, sizeof buf, "%lldx%lldx%lld:", (long long)L.g.n[0], (long long)L.g.n[1], (long long)L.g.n[2]);
    k += buf;
    for (int b = 0; b < L.dev.nb; ++b) {
      snprintf(buf, sizeof buf, "%d.%d.%lld,", L.dev.blk[b].op, L.dev.blk[b].type, (long long)L.dev.blk[b].M);
      k += buf;
    }
    k += ';';
  }
  return k;
}

static sip_status rebuild_plan(sip_handle *h, const sip_tuning *t) {
  std::vector<InstLayout> L = h->layouts0;
  h->lev[0].release();
  h->lev[0] = Plan();
  h->warm_next = h->warm_pen = false;
  return plan_build(h->lev[0], L, h->opts.dtype, true, h->batch > 0, false, t);
}

// Milliseconds per iteration of a plan built with knobs t, on model m_dev:
// the best of two timed runs of a few iterations (after one that captures
// the graph), each from the initial state.
static sip_status measure_plan(sip_handle *h, const sip_tuning &t, const void *m_dev, cudaStream_t st,
                               double *ms_iter, sip_tuning *built) {
  Plan T;
  std::vector<InstLayout> L = h->layouts0;
  sip_status s = plan_build(T, L, h->opts.dtype, true, h->batch > 0, false, &t);
  if (!s && h->batch)
    s = cudaMemcpyAsync(T.m_pack, m_dev, (size_t)T.pack_off[T.ninst] * esz(T.dtype), cudaMemcpyDeviceToDevice, st)
            ? fail(SIP_ERR_CUDA, "model copy failed")
            : SIP_OK;
  else if (!s)
    s = plan_set_m(T, 0, m_dev, st);
  const int K = T.max_iter < 10 ? T.max_iter : 10;
  double best = 1e300;
  for (int rep = 0; rep < 3 && !s; ++rep) {
    s = plan_prepare(T, st, false);
    if (s) break;
    if (cudaEventRecord(h->ev0, st) != cudaSuccess) s = fail(SIP_ERR_CUDA, "event record failed");
    if (!s) s = run_iterations(T, st, h->cap, K, false, h->pinned, nullptr);
    if (!s && cudaEventRecord(h->ev1, st) != cudaSuccess) s = fail(SIP_ERR_CUDA, "event record failed");
    if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = fail(SIP_ERR_CUDA, "tuning run failed");
    float ms = 0.f;
    if (!s && rep > 0 && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess && ms < best) best = ms;
  }
  if (built) plan_tuning(T, built);
  T.release();
  *ms_iter = best / (K > 0 ? K : 1);
  return s;
}

static bool same_knobs(const sip_tuning &a, const sip_tuning &b) {
  return a.scale_n == b.scale_n && a.scale_set == b.scale_set && a.scale_sel == b.scale_sel &&
         a.scale_fin == b.scale_fin && a.exec == b.exec && a.cluster_ctas == b.cluster_ctas &&
         a.select_window == b.select_window && a.stage_rhs == b.stage_rhs;
}

static sip_status tune_handle(sip_handle *h, const void *m_dev, cudaStream_t st) {
  h->tuned = true;
  const std::string key = tune_key(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      sip_tuning cur;
      plan_tuning(h->lev[0], &cur);
      sip_status s = same_knobs(cur, it->second) ? SIP_OK : rebuild_plan(h, &it->second);
      h->report = it->second;
      h->report.from_cache = 1;
      return s;
    }
  }
  sip_tuning base;
  plan_tuning(h->lev[0], &base);
  double ms0 = 0.0;
  sip_status s = measure_plan(h, base, m_dev, st, &ms0, nullptr);
  if (s) return s;
  sip_tuning best = base;
  double best_ms = ms0;
  int tried = 1;
  auto consider = [&](sip_tuning t) -> sip_status {
    sip_tuning built;
    double ms = 0.0;
    sip_status e = measure_plan(h, t, m_dev, st, &ms, &built);
    if (e) return e;
    ++tried;
    if (ms < 0.97 * best_ms) {  // a clear gain only: measurements carry a few % of noise
      best = built;
      best_ms = ms;
    }
    return SIP_OK;
  };
  // 1. execution form: the cluster form for small instances
  int64_t max_n = 0;
  bool blur = false, card = false;
  for (const InstLayout &L : h->layouts0) {
    if (L.dev.N > max_n) max_n = L.dev.N;
    blur = blur || L.dev.bl_R != 0;
    for (int b = 0; b < L.dev.nb; ++b) card = card || L.dev.blk[b].type == BT_CARD;
  }
  if (h->opts.exec == SIP_EXEC_AUTO && !blur && max_n <= 65536) {
    for (int c : {4, 8, 16}) {
      sip_tuning t = best;
      t.exec = SIP_EXEC_CLUSTER;
      t.cluster_ctas = c;
      if ((s = consider(t))) return s;
    }
  }
  // 2. work-item sizes per launch kind (graph form), 3. the top-k window,
  // 4. the staged right-hand side
  if (best.exec != SIP_EXEC_CLUSTER) {
    double sip_tuning::*knob[4] = {&sip_tuning::scale_n, &sip_tuning::scale_set, &sip_tuning::scale_sel,
                                   &sip_tuning::scale_fin};
    for (auto k : knob) {
      const double v0 = best.*k;
      for (double f : {0.5, 2.0, 0.25}) {
        sip_tuning t = best;
        t.*k = v0 * f;
        if ((s = consider(t))) return s;
      }
    }
    if (card) {
      sip_tuning t = best;
      t.select_window = 1 - best.select_window;
      if ((s = consider(t))) return s;
    }
    if (best.stage_rhs) {
      sip_tuning t = best;
      t.stage_rhs = 0;
      if ((s = consider(t))) return s;
    }
  }
  if (!same_knobs(best, base) && (s = rebuild_plan(h, &best))) return s;
  plan_tuning(h->lev[0], &h->report);
  h->report.tuned = 1;
  h->report.from_cache = 0;
  h->report.candidates = tried;
  h->report.ms_default = ms0;
  h->report.ms_best = best_ms;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = h->report;
  return SIP_OK;
}

// BF16 storage trial (sip_options.store_bf16): n values of a plan-owned
// binary32 array rounded to bfloat16 in place.
static sip_status round_bf16(const Plan &P, void *a, int64_t n, cudaStream_t st) {
  if (P.h_insts.empty() || !P.h_insts[0].bf16) return SIP_OK;
  CKH(launch_round_bf16(Launch{P.dtype, st}, a, n));
  return SIP_OK;
}

static sip_status project_impl(sip_handle *h, const void *m_dev, void *x_dev, cudaStream_t st, sip_info *info) {
  const NvtxRange range("sip_project");
  Plan &F = h->lev[0];
  const sip_options &o = h->opts;
  const size_t W = esz(o.dtype);
  const InstDev &df = F.h_insts[0];
  KernelTimer *tm = h->timing ? &h->timer : nullptr;
  CKH(cudaEventRecord(h->ev0, st));
  if (h->levels > 1) {
    // Algorithm ML-PARSDMM: models restricted level by level; the coarsest
    // level starts from zeros, every finer one from the interpolated x, y_i,
    // v_i of the level below
    const Launch L{o.dtype, st};
    for (int l = 1; l < h->levels; ++l) {
      int64_t fd[3], cd[3];
      int stag;
      part_dims(h->lev[l - 1].layouts[0].g, SEG_I, fd, stag);
      part_dims(h->lev[l].layouts[0].g, SEG_I, cd, stag);
      CKH(launch_restrict(L, fd, cd, l == 1 ? m_dev : h->lev[l - 1].h_insts[0].m, (void *)h->lev[l].h_insts[0].m));
    }
    for (int l = 1; l < h->levels; ++l) {
      const InstDev &dl = h->lev[l].h_insts[0];
      if (sip_status s = round_bf16(h->lev[l], (void *)dl.m, dl.N, st)) return s;
    }
    for (int l = h->levels - 1; l >= 1; --l) {
      const NvtxRange lr("sip: coarse level");
      Plan &C = h->lev[l];
      sip_status s = plan_prepare(C, st, l < h->levels - 1);
      if (!s) s = run_iterations(C, st, h->cap, C.max_iter, o.stop != 0, h->pinned, tm);
      if (!s) s = prolong_state(C, h->lev[l - 1], st);
      if (!s) {
        const Plan &Fl = h->lev[l - 1];
        const int64_t M = Fl.layouts[0].Mtot;
        s = round_bf16(Fl, Fl.h_insts[0].y, M, st);
        if (!s) s = round_bf16(Fl, Fl.h_insts[0].v, M, st);
      }
      if (s) return s;
    }
    sip_status s = plan_set_m(F, 0, m_dev, st);
    if (!s) s = round_bf16(F, (void *)df.m, df.N, st);
    if (!s) s = plan_prepare(F, st, true);
    if (s) return s;
  } else {
    sip_status s = plan_set_m(F, 0, m_dev, st);
    if (!s) s = round_bf16(F, (void *)df.m, df.N, st);
    if (s) return s;
    const int nb = df.nb;
    if (o.rho_schedule)
      CKH(cudaMemcpyAsync((void *)df.rho_sched, o.rho_schedule, (size_t)o.max_iter * nb * 8, cudaMemcpyHostToDevice, st));
    if (o.gamma_schedule)
      CKH(cudaMemcpyAsync((void *)df.gamma_sched, o.gamma_schedule, (size_t)o.max_iter * nb * 8,
                          cudaMemcpyHostToDevice, st));
    if ((s = plan_prepare(F, st, h->warm_next))) return s;
    if (h->warm_next && h->warm_pen && !o.rho_schedule && (s = load_penalties(h, F, st))) return s;
    if (h->warm_next && h->warm_k0 && !o.rho_schedule && (s = load_adapt_state(h, F, st))) return s;
    h->warm_next = h->warm_pen = h->warm_k0 = false;
  }
  sip_status s = run_iterations(F, st, h->cap, F.max_iter, o.stop != 0, h->pinned, tm);
  if (s) return s;
  CKH(cudaMemcpyAsync(x_dev, df.x, (size_t)df.N * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaEventRecord(h->ev1, st));
  const bool sync = info || o.trace || tm;
  if (!sync) return SIP_OK;
  CKH(cudaStreamSynchronize(st));
  uint32_t ctrl[8];
  CKH(cudaMemcpy(ctrl, F.d_ctrl, sizeof ctrl, cudaMemcpyDeviceToHost));
  if (ctrl[2] != 0)
    return device_error(ctrl);
  InstScal sc;
  CKH(cudaMemcpy(&sc, F.d_scal, sizeof sc, cudaMemcpyDeviceToHost));
  if (o.trace) CKH(cudaMemcpy(o.trace, df.trace, (size_t)o.max_iter * df.trace_w * 8, cudaMemcpyDeviceToHost));
  if (info) {
    memset(info, 0, sizeof *info);
    info->iters = sc.iters;
    info->cg_steps_total = sc.cg_total;
    info->stop_reason = sc.stop_reason;
    info->nblocks = df.nb;
    info->r_evol = sc.r_evol;
    for (int b = 0; b < df.p; ++b) {
      info->r_feas[b] = sc.r_feas[b];
      info->sigma[b] = sc.sigma[b];
      info->k[b] = sc.kcard[b];
    }
    for (int b = 0; b < df.nb; ++b) {
      info->rho[b] = sc.rho[b];
      info->gamma[b] = sc.gamma[b];
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
    info->window_hits = sc.win_hits;
  }
  if (sc.stop_reason < 0) return fail(SIP_ERR_NONFINITE, "the model holds NaN or Inf");
  return SIP_OK;
}

// Warm start: the handle's x, y and v (y and v: every block's rows, block
// order, the identity block last in the paper's form).
static sip_status state_check(const sip_handle *h) {
  if (!h) return fail(SIP_ERR_INVALID_ARG, "handle is NULL");
  if (h->batch) return fail(SIP_ERR_INVALID_ARG, "batched handle: no single state");
  if (h->levels > 1) return fail(SIP_ERR_INVALID_ARG, "multilevel handle: each level has its own state");
  return SIP_OK;
}

int64_t sip_state_rows(const sip_handle *h) {
  if (state_check(h)) return -1;
  return h->lev[0].layouts[0].Mtot;
}

sip_status sip_get_state(sip_handle *h, void *x_dev, void *y_dev, void *v_dev, void *stream) {
  if (sip_status s = state_check(h)) return h ? keep(h, s) : s;
  const InstDev &d = h->lev[0].h_insts[0];
  const size_t W = esz(h->opts.dtype), M = (size_t)h->lev[0].layouts[0].Mtot;
  const cudaStream_t st = (cudaStream_t)stream;
  if (x_dev) CKH(cudaMemcpyAsync(x_dev, d.x, (size_t)d.N * W, cudaMemcpyDeviceToDevice, st));
  if (y_dev) CKH(cudaMemcpyAsync(y_dev, d.y, M * W, cudaMemcpyDeviceToDevice, st));
  if (v_dev) CKH(cudaMemcpyAsync(v_dev, d.v, M * W, cudaMemcpyDeviceToDevice, st));
  return SIP_OK;
}

sip_status sip_set_state(sip_handle *h, const void *x_dev, const void *y_dev, const void *v_dev, const double *rho,
                         const double *gamma, void *stream) {
  if (sip_status s = state_check(h)) return h ? keep(h, s) : s;
  if (!x_dev) return keep(h, fail(SIP_ERR_INVALID_ARG, "x_dev is NULL"));
  // a rejected or failed call leaves no warm start armed: the next
  // projection starts from zeros
  h->warm_next = false;
  const int nb = h->lev[0].h_insts[0].nb;
  h->warm_pen = rho || gamma;
  h->warm_rho.assign(nb, h->opts.rho0);
  h->warm_gamma.assign(nb, h->opts.gamma0);
  for (int b = 0; b < nb; ++b) {
    if (rho) h->warm_rho[b] = rho[b];
    if (gamma) h->warm_gamma[b] = gamma[b];
    if (!(h->warm_rho[b] > 0.0) || !std::isfinite(h->warm_rho[b]) || !(h->warm_gamma[b] > 0.0) ||
        !(h->warm_gamma[b] < 2.0)) {
      h->warm_pen = false;
      return keep(h, fail(SIP_ERR_INVALID_ARG, "block %d: rho must be finite and > 0, gamma in (0, 2)", b));
    }
  }
  const InstDev &d = h->lev[0].h_insts[0];
  const size_t W = esz(h->opts.dtype), M = (size_t)h->lev[0].layouts[0].Mtot;
  const cudaStream_t st = (cudaStream_t)stream;
  CKH(cudaMemcpyAsync(d.x, x_dev, (size_t)d.N * W, cudaMemcpyDeviceToDevice, st));
  if (y_dev)
    CKH(cudaMemcpyAsync(d.y, y_dev, M * W, cudaMemcpyDeviceToDevice, st));
  else
    CKH(cudaMemsetAsync(d.y, 0, M * W, st));
  if (v_dev)
    CKH(cudaMemcpyAsync(d.v, v_dev, M * W, cudaMemcpyDeviceToDevice, st));
  else
    CKH(cudaMemsetAsync(d.v, 0, M * W, st));
  {
    const Plan &F0 = h->lev[0];
    if (sip_status s2 = round_bf16(F0, d.y, (int64_t)M, st)) return keep(h, s2);
    if (sip_status s2 = round_bf16(F0, d.v, (int64_t)M, st)) return keep(h, s2);
  }
  h->warm_next = true;
  return SIP_OK;
}

static sip_status adapt_state_check(const sip_handle *h) {
  if (sip_status s = state_check(h)) return s;
  const InstDev &d = h->lev[0].h_insts[0];
  if (!h->opts.adapt || h->dykstra) return fail(SIP_ERR_INVALID_ARG, "the handle does not adapt rho");
  if (!d.k0_ring)
    return fail(SIP_ERR_INVALID_ARG, "adapt state needs adapt_every < evol_hist (x^{k0} in the history ring)");
  return SIP_OK;
}

sip_status sip_get_adapt_state(sip_handle *h, void *vhat_dev, void *y_dev, void *v_dev, void *xk0_dev, int *have,
                               void *stream) {
  if (sip_status s = adapt_state_check(h)) return h ? keep(h, s) : s;
  if (!have) return keep(h, fail(SIP_ERR_INVALID_ARG, "have is NULL"));
  const Plan &F = h->lev[0];
  const InstDev &d = F.h_insts[0];
  const size_t W = esz(h->opts.dtype), M = (size_t)F.layouts[0].Mtot, N = (size_t)d.N;
  const cudaStream_t st = (cudaStream_t)stream;
  CKH(cudaStreamSynchronize(st));
  InstScal sc;
  CKH(cudaMemcpy(&sc, F.d_scal, sizeof sc, cudaMemcpyDeviceToHost));
  *have = 0;
  // the last adapt iteration k0 <= iters (k0 % adapt_every == 1 % adapt_every)
  const int ae = d.adapt_every, H = d.hist;
  int k0 = sc.iters;
  while (k0 >= 1 && k0 % ae != 1 % ae) --k0;
  if (!sc.have_k0 || k0 < 1) return SIP_OK;
  if (vhat_dev) CKH(cudaMemcpyAsync(vhat_dev, d.k0vh, M * W, cudaMemcpyDeviceToDevice, st));
  if (y_dev) CKH(cudaMemcpyAsync(y_dev, d.k0y, M * W, cudaMemcpyDeviceToDevice, st));
  if (v_dev) CKH(cudaMemcpyAsync(v_dev, d.k0v, M * W, cudaMemcpyDeviceToDevice, st));
  if (xk0_dev)
    CKH(cudaMemcpyAsync(xk0_dev, (const char *)d.ring + (size_t)(k0 % H) * N * W, N * W, cudaMemcpyDeviceToDevice,
                        st));
  CKH(cudaStreamSynchronize(st));
  *have = 1;
  return SIP_OK;
}

sip_status sip_set_adapt_state(sip_handle *h, const void *vhat_dev, const void *y_dev, const void *v_dev,
                               const void *xk0_dev, void *stream) {
  if (sip_status s = adapt_state_check(h)) return h ? keep(h, s) : s;
  if (!vhat_dev || !y_dev || !v_dev || !xk0_dev) return keep(h, fail(SIP_ERR_INVALID_ARG, "NULL array"));
  h->warm_k0 = false;
  const Plan &F = h->lev[0];
  const size_t W = esz(h->opts.dtype), M = (size_t)F.layouts[0].Mtot, N = (size_t)F.h_insts[0].N;
  if (!h->k0_stage && (hook_alloc_fails() || cudaMalloc(&h->k0_stage, (3 * M + N) * W) != cudaSuccess)) {
    cudaGetLastError();
    h->k0_stage = nullptr;
    return keep(h, fail(SIP_ERR_OOM, "adapt state staging: device allocation failed"));
  }
  const cudaStream_t st = (cudaStream_t)stream;
  char *dst = (char *)h->k0_stage;
  CKH(cudaMemcpyAsync(dst, vhat_dev, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync(dst + M * W, y_dev, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync(dst + 2 * M * W, v_dev, M * W, cudaMemcpyDeviceToDevice, st));
  CKH(cudaMemcpyAsync(dst + 3 * M * W, xk0_dev, N * W, cudaMemcpyDeviceToDevice, st));
  h->warm_k0 = true;
  return SIP_OK;
}

sip_status sip_project(sip_handle *h, const void *m_dev, void *x_dev, void *stream, sip_info *info) {
  if (!h) return fail(SIP_ERR_INVALID_ARG, "handle is NULL");
  if (h->batch) return keep(h, fail(SIP_ERR_INVALID_ARG, "batched handle: use sip_batch_project"));
  if (!m_dev || !x_dev) return keep(h, fail(SIP_ERR_INVALID_ARG, "m_dev / x_dev is NULL"));
  h->err.clear();
  if (h->opts.tune && !h->tuned && tunable(h) && !h->opts.rho_schedule && !h->opts.gamma_schedule &&
      !h->opts.trace && !h->warm_next) {
    if (sip_status s = tune_handle(h, m_dev, (cudaStream_t)stream)) return keep(h, s);
  }
  return keep(h, project_impl(h, m_dev, x_dev, (cudaStream_t)stream, info));
}

// ----------------------------------------------------------------------------
// per-kernel timing
// ----------------------------------------------------------------------------
static const char *kKernelNames[KT_COUNT] = {"rhs",   "cg_w0", "cg_step", "setpass", "select",
                                             "ties",  "final", "tail",    "cg_last"};

const char *sip_kernel_name(int i) { return (i >= 0 && i < KT_COUNT) ? kKernelNames[i] : ""; }

sip_status sip_get_tuning(const sip_handle *h, sip_tuning *out) {
  if (!h || !out) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  *out = h->report;
  sip_tuning k;
  plan_tuning(h->lev[0], &k);
  out->scale_n = k.scale_n;
  out->scale_set = k.scale_set;
  out->scale_sel = k.scale_sel;
  out->scale_fin = k.scale_fin;
  out->exec = k.exec;
  out->cluster_ctas = k.cluster_ctas;
  out->select_window = k.select_window;
  out->stage_rhs = k.stage_rhs;
  return SIP_OK;
}

sip_status sip_set_tuning(sip_handle *h, const sip_tuning *in) {
  if (!h || !in) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  if (!tunable(h)) return keep(h, fail(SIP_ERR_INVALID_ARG, "multilevel and parallel-Dykstra handles are not tunable"));
  for (double v : {in->scale_n, in->scale_set, in->scale_sel, in->scale_fin})
    if (!(v >= 1.0 / 16 && v <= 16.0)) return keep(h, fail(SIP_ERR_INVALID_ARG, "scales must lie in [1/16, 16]"));
  if (in->exec != SIP_EXEC_GRAPH && in->exec != SIP_EXEC_CLUSTER)
    return keep(h, fail(SIP_ERR_INVALID_ARG, "exec must be SIP_EXEC_GRAPH or SIP_EXEC_CLUSTER"));
  if (in->exec == SIP_EXEC_CLUSTER && in->cluster_ctas != 0 && in->cluster_ctas != 1 && in->cluster_ctas != 2 &&
      in->cluster_ctas != 4 && in->cluster_ctas != 8 && in->cluster_ctas != 16)
    return keep(h, fail(SIP_ERR_INVALID_ARG, "cluster_ctas must be 0, 1, 2, 4, 8 or 16"));
  if ((in->select_window != 0 && in->select_window != 1) || (in->stage_rhs != 0 && in->stage_rhs != 1))
    return keep(h, fail(SIP_ERR_INVALID_ARG, "select_window and stage_rhs must be 0 or 1"));
  h->tuned = true;  // the caller's knobs replace any tuning
  memset(&h->report, 0, sizeof h->report);
  return keep(h, rebuild_plan(h, in));
}

sip_status sip_test_hook(int hook, int64_t value) {
  if (value < 0) return fail(SIP_ERR_INVALID_ARG, "hook value must be >= 0");
  switch (hook) {
    case SIP_HOOK_FAIL_ALLOC:
      if (value > (1 << 30)) return fail(SIP_ERR_INVALID_ARG, "hook value too large");
      g_hooks.fail_alloc = (int)value;
      return SIP_OK;
    case SIP_HOOK_BARRIER_EXTRA:
      if (value > (1 << 20)) return fail(SIP_ERR_INVALID_ARG, "hook value too large");
      g_hooks.bar_extra = (uint32_t)value;
      return SIP_OK;
    case SIP_HOOK_BARRIER_SPINS:
      if (value > (INT64_C(1) << 40)) return fail(SIP_ERR_INVALID_ARG, "hook value too large");
      g_hooks.bar_spins = (long long)value;
      return SIP_OK;
    default:
      return fail(SIP_ERR_INVALID_ARG, "unknown hook %d", hook);
  }
}

sip_status sip_set_timing(sip_handle *h, int on) {
  if (!h) return fail(SIP_ERR_INVALID_ARG, "handle is NULL");
  h->timing = on != 0;
  h->timer.reset();
  return SIP_OK;
}

sip_status sip_kernel_times(const sip_handle *h, double *ms, int64_t *launches, double *bytes_per_launch) {
  if (!h) return fail(SIP_ERR_INVALID_ARG, "handle is NULL");
  const InstLayout &L = h->lev[0].layouts[0];
  const InstDev &d = L.dev;
  const double W = (double)esz(h->opts.dtype), N = (double)d.N, Mp = (double)L.Mtot;
  double Mpw = 0.0, Mms = 0.0, Msel = 0.0;
  for (int b = 0; b < d.nb; ++b) {
    const int t = d.blk[b].type;
    if (t == BT_BOUNDS || t == BT_DIST) Mpw += (double)d.blk[b].M;
    if (t == BT_L1 || t == BT_L2 || t == BT_CARD) Mms += (double)d.blk[b].M;
    if (t == BT_L1 || t == BT_CARD) Msel += (double)d.blk[b].M;
  }
  const double ad = (h->opts.adapt && !h->opts.rho_schedule) ? 1.0 / h->opts.adapt_every : 0.0;
  double bytes[KT_COUNT] = {};
  bytes[KT_RHS] = W * (2 * Mp + 2 * N + (d.alg1 ? 0 : N));
  bytes[KT_CG_W0] = W * 2 * N;   // read r, write w = C r
  bytes[KT_CG_STEP] = W * 10 * N;  // read x, p, r, w, s; write x, p, r, w, s
  bytes[KT_SETPASS] = W * (N + 2 * Mp + 2 * Mpw + Mms + (d.alg1 ? N : 0) + 2 * N + ad * (4 * Mp + 2 * Mpw));
  bytes[KT_SELECT] = W * Msel;
  bytes[KT_TIES] = 0.0;
  bytes[KT_FINAL] = W * (3 * Mms + ad * 4 * Mms);
  bytes[KT_TAIL] = 0.0;
  bytes[KT_CG_LAST] = W * 4 * N;  // read r, p, x; write x
  for (int c = 0; c < KT_COUNT; ++c) {
    if (ms) ms[c] = h->timer.ms[c];
    if (launches) launches[c] = h->timer.launches[c];
    if (bytes_per_launch) bytes_per_launch[c] = bytes[c];
  }
  return SIP_OK;
}

// ----------------------------------------------------------------------------
// single-step entry points
// ----------------------------------------------------------------------------
int64_t sip_op_rows(const sip_grid *grid, int op) {
  if (check_grid_op(grid, op) != SIP_OK) return -1;
  return op_rows(grid_desc(*grid), op);
}

sip_status sip_apply_op(const sip_grid *grid, int op, int dtype, const void *x_dev, void *s_dev, void *stream) {
  sip_status st = check_grid_op(grid, op);
  if (st) return st;
  if (dtype != SIP_F64 && dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "unknown dtype");
  if (!x_dev || !s_dev) return fail(SIP_ERR_INVALID_ARG, "NULL buffer");
  const GridDesc g = grid_desc(*grid);
  DevCopy<InstDev> d;
  CKH(d.make(op_inst(g, op)));
  CKH(launch_apply_op(Launch{dtype, (cudaStream_t)stream}, d.p, x_dev, s_dev, op_rows(g, op)));
  CKH(cudaStreamSynchronize((cudaStream_t)stream));
  return SIP_OK;
}

sip_status sip_apply_op_t(const sip_grid *grid, int op, int dtype, const void *s_dev, void *x_dev, void *stream) {
  sip_status st = check_grid_op(grid, op);
  if (st) return st;
  if (dtype != SIP_F64 && dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "unknown dtype");
  if (!x_dev || !s_dev) return fail(SIP_ERR_INVALID_ARG, "NULL buffer");
  const GridDesc g = grid_desc(*grid);
  DevCopy<InstDev> d;
  CKH(d.make(op_inst(g, op)));
  CKH(launch_apply_op_t(Launch{dtype, (cudaStream_t)stream}, d.p, s_dev, x_dev, g.N()));
  CKH(cudaStreamSynchronize((cudaStream_t)stream));
  return SIP_OK;
}

sip_status sip_system_apply(const sip_grid *grid, const int *ops, const double *rhos, int nops, double c_identity,
                            int dtype, const void *x_dev, void *out_dev, void *stream) {
  sip_status st = check_grid_op(grid, SIP_OP_I);
  if (st) return st;
  if (dtype != SIP_F64 && dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "unknown dtype");
  if (!x_dev || !out_dev || (nops > 0 && (!ops || !rhos)) || nops < 0)
    return fail(SIP_ERR_INVALID_ARG, "NULL buffer or bad nops");
  const GridDesc g = grid_desc(*grid);
  InstScal sc;
  memset(&sc, 0, sizeof sc);
  double c0 = c_identity, cz = 0, cx = 0, cy = 0;
  for (int i = 0; i < nops; ++i) {
    if ((st = check_grid_op(grid, ops[i]))) return st;
    switch (ops[i]) {
      case SIP_OP_I: c0 += rhos[i]; break;
      case SIP_OP_DZ: cz += rhos[i]; break;
      case SIP_OP_DX: cx += rhos[i]; break;
      case SIP_OP_DY: cy += rhos[i]; break;
      default: cz += rhos[i]; cx += rhos[i]; if (g.ndim == 3) cy += rhos[i]; break;
    }
  }
  sc.c0 = c0;
  sc.cz = cz / (g.h[0] * g.h[0]);
  sc.cx = cx / (g.h[1] * g.h[1]);
  sc.cy = cy / (g.h[2] * g.h[2]);
  sc.cf[0] = (float)sc.c0;
  sc.cf[1] = (float)sc.cz;
  sc.cf[2] = (float)sc.cx;
  sc.cf[3] = (float)sc.cy;
  DevCopy<InstDev> d;
  DevCopy<InstScal> ds;
  CKH(d.make(op_inst(g, SIP_OP_I)));
  CKH(ds.make(sc));
  CKH(launch_system_apply(Launch{dtype, (cudaStream_t)stream}, d.p, ds.p, x_dev, out_dev, g.N()));
  CKH(cudaStreamSynchronize((cudaStream_t)stream));
  return SIP_OK;
}

sip_status sip_project_set(const sip_set *set, int dtype, const void *w_dev, int64_t n, void *y_dev, void *stream,
                           double *scalar_out) {
  if (!set || !w_dev || !y_dev) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(SIP_ERR_INVALID_ARG, "n must be >= 1");
  if (set->scope != SIP_SCOPE_ALL) return fail(SIP_ERR_INVALID_ARG, "a single-step set applies to the whole vector");
  sip_set s = *set;
  s.op = SIP_OP_I;
  s.sigma_rel = 0.0;
  s.k_frac = 0.0;
  sip_grid g;
  memset(&g, 0, sizeof g);
  g.ndim = 2;
  g.n[0] = n;
  g.n[1] = 1;
  g.h[0] = g.h[1] = 1.0;
  sip_options o;
  sip_options_default(&o);
  o.dtype = dtype;
  o.form = SIP_FORM_DIRECT;
  o.adapt = 0;
  o.max_iter = 1;
  o.gamma0 = 1.0;
  o.rho0 = 1.0;
  o.check_every = 1 << 30;
  sip_status st = validate(&g, &s, 1, &o);
  if (st) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  Plan P;
  std::vector<InstLayout> L{make_layout(grid_desc(g), &s, 1, o)};
  if ((st = plan_build(P, L, dtype, false))) return st;
  struct Rel {
    Plan &p;
    ~Rel() { p.release(); }
  } rel{P};
  const InstDev &d = P.h_insts[0];
  const Launch Ln{dtype, cs};
  if ((st = plan_set_m(P, 0, w_dev, cs))) return st;
  if ((st = plan_prepare(P, cs, false))) return st;
  CKH(cudaMemcpyAsync(d.x, w_dev, (size_t)n * esz(dtype), cudaMemcpyDeviceToDevice, cs));
  CKH(launch_setpass(Ln, P.d_tset, P.nt_set, P.d_insts, P.d_scal, P.d_jscal, P.d_jobs, P.one));
  if (P.nt_sel)
    for (int pass = 0; pass < select_passes(dtype); ++pass)
      CKH(launch_select(Ln, P.d_tsel, P.nt_sel, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_hcnt, P.d_hs1, P.d_hs2,
                        P.d_hs3, (int64_t)P.njobs * kBins, pass, P.one));
  if (P.any_card) CKH(launch_ties(Ln, P.d_tfin, P.nt_fin, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_ties, P.one));
  if (P.nt_fin) CKH(launch_final(Ln, P.d_tfin, P.nt_fin, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_ties, P.one));
  CKH(cudaMemcpyAsync(y_dev, d.y, (size_t)n * esz(dtype), cudaMemcpyDeviceToDevice, cs));
  CKH(cudaStreamSynchronize(cs));
  if (scalar_out) {
    *scalar_out = 0.0;
    if (s.type == SIP_SET_L2) {
      InstScal sc;
      CKH(cudaMemcpy(&sc, P.d_scal, sizeof sc, cudaMemcpyDeviceToHost));
      *scalar_out = sc.l2scale[0];
    } else if (s.type == SIP_SET_L1 || s.type == SIP_SET_CARD) {
      JobScal js;
      CKH(cudaMemcpy(&js, P.d_jscal + d.blk[0].job_w, sizeof js, cudaMemcpyDeviceToHost));
      if (js.mode == JM_SELECT) *scalar_out = s.type == SIP_SET_L1 ? js.theta : js.kval;
    }
  }
  return SIP_OK;
}

sip_status sip_op_norm(const sip_grid *grid, int op, int type, int dtype, const void *m_dev, void *stream,
                       double *out) {
  if (!out || !m_dev) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  if (type != SIP_SET_L1 && type != SIP_SET_L2) return fail(SIP_ERR_INVALID_ARG, "type must be L1 or L2");
  sip_set s;
  memset(&s, 0, sizeof s);
  s.op = op;
  s.type = type;
  s.sigma_rel = 1.0;
  sip_options o;
  sip_options_default(&o);
  o.dtype = dtype;
  o.form = SIP_FORM_DIRECT;
  o.adapt = 0;
  o.max_iter = 1;
  sip_status st = validate(grid, &s, 1, &o);
  if (st) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  Plan P;
  std::vector<InstLayout> L{make_layout(grid_desc(*grid), &s, 1, o)};
  if ((st = plan_build(P, L, dtype, false))) return st;
  struct Rel {
    Plan &p;
    ~Rel() { p.release(); }
  } rel{P};
  if ((st = plan_set_m(P, 0, m_dev, cs))) return st;
  if ((st = plan_prepare(P, cs, false))) return st;
  CKH(cudaStreamSynchronize(cs));
  InstScal sc;
  CKH(cudaMemcpy(&sc, P.d_scal, sizeof sc, cudaMemcpyDeviceToHost));
  *out = sc.sigma[0];
  return SIP_OK;
}

// ----------------------------------------------------------------------------
// batched (ragged) projections
// ----------------------------------------------------------------------------
sip_status sip_batch_create(int count, const sip_grid *grids, const sip_set *sets, const int *nsets,
                            const sip_options *opts, sip_handle **out) {
  if (!out) return fail(SIP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1) return fail(SIP_ERR_INVALID_ARG, "count must be >= 1");
  if (!grids || !sets || !nsets || !opts) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  if (opts->levels != 1) return fail(SIP_ERR_INVALID_ARG, "batched projections are single-level");
  if (opts->rho_schedule || opts->gamma_schedule || opts->trace)
    return fail(SIP_ERR_INVALID_ARG, "schedules and traces are per-handle, not batched");
  std::vector<InstLayout> L;
  L.reserve(count);
  int64_t so = 0;
  for (int i = 0; i < count; ++i) {
    sip_status st = validate(&grids[i], sets + so, nsets[i], opts);
    if (st) return fail(st, "instance %d: %s", i, g_err.c_str());
    L.push_back(make_layout(grid_desc(grids[i]), sets + so, nsets[i], *opts));
    so += nsets[i];
  }
  sip_handle *h = new (std::nothrow) sip_handle();
  if (!h) return fail(SIP_ERR_OOM, "host allocation failed");
  h->opts = *opts;
  h->grid = grids[0];
  h->batch = count;
  h->layouts0 = L;
  memset(&h->report, 0, sizeof h->report);
  sip_status st = plan_build(h->lev[0], L, opts->dtype, true, true);
  if (st) {
    sip_destroy(h);
    return st;
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&h->pinned, sizeof(int32_t)) != cudaSuccess || cudaEventCreate(&h->ev0) != cudaSuccess ||
      cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    sip_destroy(h);
    return fail(SIP_ERR_CUDA, "stream/event set-up failed");
  }
  *out = h;
  return SIP_OK;
}

int64_t sip_batch_offset(const sip_handle *h, int i) {
  if (!h || !h->batch || i < 0 || i > h->batch) return -1;
  return h->lev[0].pack_off[i];
}

sip_status sip_batch_project(sip_handle *h, const void *m_dev, void *x_dev, void *stream, sip_info *infos) {
  if (!h || !h->batch) return fail(SIP_ERR_INVALID_ARG, "not a batched handle");
  if (!m_dev || !x_dev) return keep(h, fail(SIP_ERR_INVALID_ARG, "m_dev / x_dev is NULL"));
  h->err.clear();
  if (h->opts.tune && !h->tuned && tunable(h)) {
    if (sip_status s = tune_handle(h, m_dev, (cudaStream_t)stream)) return keep(h, s);
  }
  Plan &P = h->lev[0];
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)P.pack_off[P.ninst] * esz(P.dtype);
  KernelTimer *tm = h->timing ? &h->timer : nullptr;
  auto run = [&]() -> sip_status {
    CKH(cudaEventRecord(h->ev0, st));
    CKH(cudaMemcpyAsync(P.m_pack, m_dev, bytes, cudaMemcpyDeviceToDevice, st));
    if (sip_status s0 = round_bf16(P, P.m_pack, (int64_t)P.pack_off[P.ninst], st)) return s0;
    sip_status s = plan_prepare(P, st, false);
    if (!s) s = run_iterations(P, st, h->cap, P.max_iter, h->opts.stop != 0, h->pinned, tm);
    if (s) return s;
    CKH(cudaMemcpyAsync(x_dev, P.x_pack, bytes, cudaMemcpyDeviceToDevice, st));
    CKH(cudaEventRecord(h->ev1, st));
    if (!infos && !tm) return SIP_OK;
    CKH(cudaStreamSynchronize(st));
    uint32_t ctrl[8];
    CKH(cudaMemcpy(ctrl, P.d_ctrl, sizeof ctrl, cudaMemcpyDeviceToHost));
    if (ctrl[2] != 0)
      return device_error(ctrl);
    if (!infos) return SIP_OK;
    std::vector<InstScal> sc(P.ninst);
    CKH(cudaMemcpy(sc.data(), P.d_scal, P.ninst * sizeof(InstScal), cudaMemcpyDeviceToHost));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    bool nonfinite = false;
    for (int i = 0; i < P.ninst; ++i) {
      const InstDev &d = P.h_insts[i];
      sip_info &f = infos[i];
      memset(&f, 0, sizeof f);
      f.iters = sc[i].iters;
      f.cg_steps_total = sc[i].cg_total;
      f.stop_reason = sc[i].stop_reason;
      f.nblocks = d.nb;
      f.r_evol = sc[i].r_evol;
      for (int b = 0; b < d.p; ++b) {
        f.r_feas[b] = sc[i].r_feas[b];
        f.sigma[b] = sc[i].sigma[b];
        f.k[b] = sc[i].kcard[b];
      }
      for (int b = 0; b < d.nb; ++b) {
        f.rho[b] = sc[i].rho[b];
        f.gamma[b] = sc[i].gamma[b];
      }
      f.ms = ms;
      f.window_hits = sc[i].win_hits;
      if (sc[i].stop_reason < 0) nonfinite = true;
    }
    if (nonfinite) return fail(SIP_ERR_NONFINITE, "a model holds NaN or Inf");
    return SIP_OK;
  };
  return keep(h, run());
}

// ----------------------------------------------------------------------------
// parallel Dykstra baseline
// ----------------------------------------------------------------------------
sip_status sip_dykstra_create(const sip_grid *grid, const sip_set *sets, int nsets, const sip_options *inner,
                              sip_handle **out) {
  if (!out) return fail(SIP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sip_status st = validate(grid, sets, nsets, inner);
  if (st) return st;
  for (int i = 0; i < nsets; ++i)
    if (sets[i].sigma_rel != 0.0) return fail(SIP_ERR_INVALID_ARG, "set %d: Dykstra's sets take absolute radii", i);
  std::vector<sip_grid> grids(nsets, *grid);
  std::vector<int> ns(nsets, 1);
  sip_handle *h = nullptr;
  if ((st = sip_batch_create(nsets, grids.data(), sets, ns.data(), inner, &h))) return st;
  h->dykstra = true;
  h->sets.assign(sets, sets + nsets);
  const size_t bytes = (size_t)grid_desc(*grid).N() * esz(inner->dtype);
  if (cudaMalloc(&h->dk_x, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->dk_x = nullptr;
    sip_destroy(h);
    return fail(SIP_ERR_OOM, "device allocation failed");
  }
  *out = h;
  return SIP_OK;
}

sip_status sip_dykstra_project(sip_handle *h, const void *m_dev, void *x_dev, int sweeps, void *stream,
                               sip_dykstra_info *info) {
  if (!h || !h->dykstra) return fail(SIP_ERR_INVALID_ARG, "not a Dykstra handle");
  if (!m_dev || !x_dev || sweeps < 1) return keep(h, fail(SIP_ERR_INVALID_ARG, "NULL buffer or sweeps < 1"));
  h->err.clear();
  Plan &P = h->lev[0];
  cudaStream_t st = (cudaStream_t)stream;
  const int p = P.ninst;
  const int64_t N = P.h_insts[0].N;
  const size_t W = esz(P.dtype);
  auto run = [&]() -> sip_status {
    if (info) memset(info, 0, sizeof *info);
    CKH(cudaEventRecord(h->ev0, st));
    for (int i = 0; i < p; ++i)  // v_i = m
      CKH(cudaMemcpyAsync((char *)P.m_pack + (size_t)i * N * W, m_dev, (size_t)N * W, cudaMemcpyDeviceToDevice, st));
    std::vector<InstScal> sc(p);
    for (int sw = 0; sw < sweeps; ++sw) {
      sip_status s = plan_prepare(P, st, false);  // every sub-problem from zero state
      if (!s) s = run_iterations(P, st, h->cap, P.max_iter, h->opts.stop != 0, h->pinned, nullptr);
      if (s) return s;
      CKH(launch_dykstra_update(Launch{P.dtype, st}, P.x_pack, P.m_pack, h->dk_x, p, N));
      if (info) {
        CKH(cudaMemcpyAsync(sc.data(), P.d_scal, p * sizeof(InstScal), cudaMemcpyDeviceToHost, st));
        CKH(cudaStreamSynchronize(st));
        int64_t cg = 0;
        for (int i = 0; i < p; ++i) {
          if (sc[i].cg_total > cg) cg = sc[i].cg_total;
          if (h->sets[i].type == SIP_SET_L1) info->l1_projections += sc[i].iters;
        }
        info->cg_steps += cg;
        info->sweeps = sw + 1;
      }
    }
    CKH(cudaMemcpyAsync(x_dev, h->dk_x, (size_t)N * W, cudaMemcpyDeviceToDevice, st));
    CKH(cudaEventRecord(h->ev1, st));
    CKH(cudaStreamSynchronize(st));
    uint32_t ctrl[8];
    CKH(cudaMemcpy(ctrl, P.d_ctrl, sizeof ctrl, cudaMemcpyDeviceToHost));
    if (ctrl[2] != 0)
      return device_error(ctrl);
    if (info) cudaEventElapsedTime(&info->ms, h->ev0, h->ev1);
    return SIP_OK;
  };
  return keep(h, run());
}

sip_status sip_restrict(const sip_grid *fine, int dtype, const void *m_dev, void *mc_dev, void *stream) {
  sip_status st = check_grid_op(fine, SIP_OP_I);
  if (st) return st;
  if (!m_dev || !mc_dev) return fail(SIP_ERR_INVALID_ARG, "NULL buffer");
  const GridDesc f = grid_desc(*fine), c = grid_desc(coarse_of(*fine));
  CKH(launch_restrict(Launch{dtype, (cudaStream_t)stream}, f.n, c.n, m_dev, mc_dev));
  CKH(cudaStreamSynchronize((cudaStream_t)stream));
  return SIP_OK;
}

sip_status sip_prolong(const sip_grid *fine, int op, int dtype, const void *uc_dev, void *uf_dev, void *stream) {
  sip_status st = check_grid_op(fine, op);
  if (st) return st;
  const sip_grid cg = coarse_of(*fine);
  if ((st = check_grid_op(&cg, op))) return fail(st, "coarse grid: %s", g_err.c_str());
  if (!uc_dev || !uf_dev) return fail(SIP_ERR_INVALID_ARG, "NULL buffer");
  const GridDesc f = grid_desc(*fine), c = grid_desc(cg);
  const Launch L{dtype, (cudaStream_t)stream};
  int64_t oc = 0, of = 0;
  for (int kind : op_parts(f, op)) {
    int64_t cd[3], fd[3];
    int stag;
    part_dims(c, kind, cd, stag);
    part_dims(f, kind, fd, stag);
    CKH(launch_prolong(L, cd, fd, stag, (const char *)uc_dev + oc * esz(dtype), (char *)uf_dev + of * esz(dtype)));
    oc += part_rows(c, kind);
    of += part_rows(f, kind);
  }
  CKH(cudaStreamSynchronize((cudaStream_t)stream));
  return SIP_OK;
}

}  // extern "C"
