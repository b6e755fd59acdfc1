// C ABI of libsip.so: handle life cycle, layout of the device arena, launch
// sequencing of Algorithm PARSDMM / ML-PARSDMM, and the single-step entry
// points.  Every argument check happens here, on the host, before any
// device work; kernels assume validated layouts.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sip.h"
#include "sip_dev.cuh"
#include "sip_kernels.h"
#include "sip_host.h"

namespace sip {

thread_local std::string g_err;
TestHooks g_hooks;

bool hook_alloc_fails() {
  if (g_hooks.fail_alloc <= 0) return false;
  return --g_hooks.fail_alloc == 0;
}

sip_status fail(sip_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(SIP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static size_t esize(int dtype) { return dtype == SIP_F64 ? 8 : 4; }
static int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// ----------------------------------------------------------------------------
// grid and operator geometry
// ----------------------------------------------------------------------------
GridDesc grid_desc(const sip_grid &g) {
  GridDesc d;
  d.ndim = g.ndim;
  d.n[0] = g.n[0];
  d.n[1] = g.n[1];
  d.n[2] = g.ndim == 3 ? g.n[2] : 1;
  d.h[0] = g.h[0];
  d.h[1] = g.h[1];
  d.h[2] = g.ndim == 3 ? g.h[2] : 1.0;
  return d;
}

std::vector<int> op_parts(const GridDesc &g, int op) {
  switch (op) {
    case SIP_OP_I: return {SEG_I};
    case SIP_OP_DZ: return {SEG_DZ};
    case SIP_OP_DX: return {SEG_DX};
    case SIP_OP_DY: return {SEG_DY};
    case SIP_OP_BLUR: return {SEG_BLUR};
    default:
      if (g.ndim == 3) return {SEG_DZ, SEG_DX, SEG_DY};
      return {SEG_DZ, SEG_DX};
  }
}

int64_t part_rows(const GridDesc &g, int kind) {
  switch (kind) {
    case SEG_DZ: return (g.n[0] - 1) * g.n[1] * g.n[2];
    case SEG_DX: return g.n[0] * (g.n[1] - 1) * g.n[2];
    case SEG_DY: return g.n[0] * g.n[1] * (g.n[2] - 1);
    default: return g.N();
  }
}

int64_t op_rows(const GridDesc &g, int op) {
  int64_t m = 0;
  for (int k : op_parts(g, op)) m += part_rows(g, k);
  return m;
}

// output-grid dims (nz, nx, ny) of one part and the staggered axis
void part_dims(const GridDesc &g, int kind, int64_t d[3], int &stag) {
  d[0] = g.n[0];
  d[1] = g.n[1];
  d[2] = g.n[2];
  stag = -1;
  if (kind == SEG_DZ) { d[0] -= 1; stag = 0; }
  if (kind == SEG_DX) { d[1] -= 1; stag = 1; }
  if (kind == SEG_DY) { d[2] -= 1; stag = 2; }
}

static sip_status check_grid(const sip_grid *g) {
  if (!g) return fail(SIP_ERR_INVALID_ARG, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(SIP_ERR_INVALID_ARG, "grid.ndim must be 2 or 3 (got %d)", g->ndim);
  for (int a = 0; a < g->ndim; ++a) {
    if (g->n[a] < 1) return fail(SIP_ERR_INVALID_ARG, "grid.n[%d] = %lld < 1", a, (long long)g->n[a]);
    if (!(g->h[a] > 0.0) || !std::isfinite(g->h[a]))
      return fail(SIP_ERR_INVALID_ARG, "grid.h[%d] must be finite and > 0", a);
  }
  const GridDesc d = grid_desc(*g);
  if (d.N() >= (int64_t(1) << 31) / 4) return fail(SIP_ERR_INVALID_ARG, "grid too large (N = %lld)", (long long)d.N());
  return SIP_OK;
}

static sip_status check_op(const GridDesc &g, int op) {
  if (op < SIP_OP_I || op > SIP_OP_BLUR) return fail(SIP_ERR_INVALID_ARG, "unknown operator %d", op);
  if (op == SIP_OP_DY && g.ndim != 3) return fail(SIP_ERR_INVALID_ARG, "D_y needs a 3D grid");
  if ((op == SIP_OP_DZ || op == SIP_OP_TV) && g.n[0] < 2) return fail(SIP_ERR_INVALID_ARG, "operator needs n_z >= 2");
  if ((op == SIP_OP_DX || op == SIP_OP_TV) && g.n[1] < 2) return fail(SIP_ERR_INVALID_ARG, "operator needs n_x >= 2");
  if ((op == SIP_OP_DY || (op == SIP_OP_TV && g.ndim == 3)) && g.n[2] < 2)
    return fail(SIP_ERR_INVALID_ARG, "operator needs n_y >= 2");
  return SIP_OK;
}

static sip_status check_set(const GridDesc &g, const sip_set &s, int i) {
  sip_status st = check_op(g, s.op);
  if (st) return fail(st, "set %d: %s", i, g_err.c_str());
  if (s.op == SIP_OP_BLUR) {
    if (s.blur_axis < 0 || s.blur_axis > 2 || (s.blur_axis == 2 && g.ndim != 3))
      return fail(SIP_ERR_INVALID_ARG, "set %d: blur axis must be 0 (z), 1 (x) or 2 (y, 3D)", i);
    if (s.blur_radius < 1 || s.blur_radius > SIP_MAX_BLUR_RADIUS)
      return fail(SIP_ERR_INVALID_ARG, "set %d: blur radius must be in [1, %d]", i, SIP_MAX_BLUR_RADIUS);
    if (!s.blur_taps) return fail(SIP_ERR_INVALID_ARG, "set %d: a blur needs its taps", i);
    for (int t = 0; t <= s.blur_radius; ++t)
      if (!std::isfinite(s.blur_taps[t])) return fail(SIP_ERR_INVALID_ARG, "set %d: blur taps must be finite", i);
    if (s.scope != SIP_SCOPE_ALL) return fail(SIP_ERR_INVALID_ARG, "set %d: a blur set applies to the whole model", i);
  }
  switch (s.type) {
    case SIP_SET_BOUNDS: {
      if (std::isnan(s.lo) || std::isnan(s.hi) || (!s.lo_vec && !s.hi_vec && s.lo > s.hi))
        return fail(SIP_ERR_INVALID_ARG, "set %d: bounds need lo <= hi", i);
      if (s.lo_vec || s.hi_vec) {
        const int64_t M = op_rows(g, s.op);
        for (int64_t j = 0; j < M; ++j) {
          const double lo = s.lo_vec ? s.lo_vec[j] : s.lo, hi = s.hi_vec ? s.hi_vec[j] : s.hi;
          if (std::isnan(lo) || std::isnan(hi) || lo > hi)
            return fail(SIP_ERR_INVALID_ARG, "set %d: per-entry bounds need lo <= hi (entry %lld)", i, (long long)j);
        }
      }
      break;
    }
    case SIP_SET_L1:
    case SIP_SET_L2:
      if (!(s.sigma >= 0.0) || !std::isfinite(s.sigma)) return fail(SIP_ERR_INVALID_ARG, "set %d: sigma < 0", i);
      if (!(s.sigma_rel >= 0.0) || !std::isfinite(s.sigma_rel))
        return fail(SIP_ERR_INVALID_ARG, "set %d: sigma_rel < 0", i);
      break;
    case SIP_SET_CARD:
      if (s.k < 0) return fail(SIP_ERR_INVALID_ARG, "set %d: k < 0", i);
      if (!(s.k_frac >= 0.0) || !(s.k_frac <= 1.0)) return fail(SIP_ERR_INVALID_ARG, "set %d: k_frac not in [0, 1]", i);
      break;
    case SIP_SET_ANNULUS:
      if (!(s.lo >= 0.0) || !std::isfinite(s.lo) || !(s.hi >= s.lo))
        return fail(SIP_ERR_INVALID_ARG, "set %d: annulus needs 0 <= lo <= hi", i);
      break;
    default:
      return fail(SIP_ERR_INVALID_ARG, "set %d: unknown set type %d", i, s.type);
  }
  if (s.scope < SIP_SCOPE_ALL || s.scope > SIP_SCOPE_Y) return fail(SIP_ERR_INVALID_ARG, "set %d: unknown scope", i);
  if ((s.lo_vec || s.hi_vec) && s.type != SIP_SET_BOUNDS)
    return fail(SIP_ERR_INVALID_ARG, "set %d: per-entry vectors are for bounds sets", i);
  if (s.center_vec && (s.type != SIP_SET_L2 || s.sigma_rel != 0.0 || s.scope != SIP_SCOPE_ALL))
    return fail(SIP_ERR_INVALID_ARG, "set %d: a center goes with an absolute l2 radius on the whole set", i);
  if (s.scope != SIP_SCOPE_ALL && s.type != SIP_SET_BOUNDS) {
    if (s.op == SIP_OP_TV) return fail(SIP_ERR_INVALID_ARG, "set %d: per-line sets need a single-grid operator", i);
    if (s.sigma_rel != 0.0) return fail(SIP_ERR_INVALID_ARG, "set %d: per-line sets take absolute radii", i);
    if (s.scope == SIP_SCOPE_Y && g.ndim != 3) return fail(SIP_ERR_INVALID_ARG, "set %d: lines along y need 3D", i);
    int64_t d[3];
    int stag;
    part_dims(g, op_parts(g, s.op)[0], d, stag);
    const int64_t len = d[s.scope - 1];
    if ((s.type == SIP_SET_CARD || s.type == SIP_SET_L1) && len > SIP_MAX_LINE)
      return fail(SIP_ERR_INVALID_ARG, "set %d: lines of %lld entries exceed %d", i, (long long)len, SIP_MAX_LINE);
  }
  return SIP_OK;
}

static sip_status check_opts(const sip_options &o) {
  if (o.max_iter < 1) return fail(SIP_ERR_INVALID_ARG, "max_iter must be >= 1");
  if (o.cg_iters < 0 || o.cg_max < 1 || o.cg_iters > 1000 || o.cg_max > 1000)
    return fail(SIP_ERR_INVALID_ARG, "cg_iters in [0, 1000], cg_max in [1, 1000]");
  if (o.check_every < 1) return fail(SIP_ERR_INVALID_ARG, "check_every must be >= 1");
  if (o.evol_hist < 1 || o.evol_hist > kMaxHist) return fail(SIP_ERR_INVALID_ARG, "evol_hist must be in [1, %d]", kMaxHist);
  if (o.stop < 0 || o.stop > 2) return fail(SIP_ERR_INVALID_ARG, "stop must be 0, 1 or 2");
  if (o.adapt < 0 || o.adapt > 2) return fail(SIP_ERR_INVALID_ARG, "adapt must be 0, 1 or 2");
  if (o.adapt_every < 1) return fail(SIP_ERR_INVALID_ARG, "adapt_every must be >= 1");
  if (!(o.rho0 > 0.0) || !std::isfinite(o.rho0)) return fail(SIP_ERR_INVALID_ARG, "rho0 must be > 0");
  if (!(o.gamma0 > 0.0) || !(o.gamma0 < 2.0)) return fail(SIP_ERR_INVALID_ARG, "gamma0 must be in (0, 2)");
  if (!(o.rho_ratio_max >= 1.0)) return fail(SIP_ERR_INVALID_ARG, "rho_ratio_max must be >= 1");
  if (!(o.gamma_max > 0.0) || !(o.gamma_max < 2.0)) return fail(SIP_ERR_INVALID_ARG, "gamma_max must be in (0, 2)");
  if (o.form != SIP_FORM_ALG1 && o.form != SIP_FORM_DIRECT) return fail(SIP_ERR_INVALID_ARG, "unknown form");
  if (o.dtype != SIP_F64 && o.dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "unknown dtype");
  if (o.levels < 1 || o.levels > SIP_MAX_LEVELS) return fail(SIP_ERR_INVALID_ARG, "levels must be in [1, %d]", SIP_MAX_LEVELS);
  if (o.coarse_iter < 0) return fail(SIP_ERR_INVALID_ARG, "coarse_iter < 0");
  if (o.levels > 1 && (o.rho_schedule || o.gamma_schedule || o.trace))
    return fail(SIP_ERR_INVALID_ARG, "schedules and traces are single-level only");
  if (o.gamma_schedule && !o.rho_schedule) return fail(SIP_ERR_INVALID_ARG, "gamma_schedule needs rho_schedule");
  if (o.exec < SIP_EXEC_AUTO || o.exec > SIP_EXEC_CLUSTER) return fail(SIP_ERR_INVALID_ARG, "unknown exec mode");
  if (o.cluster_ctas != 0 && o.cluster_ctas != 1 && o.cluster_ctas != 2 && o.cluster_ctas != 4 &&
      o.cluster_ctas != 8 && o.cluster_ctas != 16)
    return fail(SIP_ERR_INVALID_ARG, "cluster_ctas must be 0, 1, 2, 4, 8 or 16");
  if (o.tune != 0 && o.tune != 1) return fail(SIP_ERR_INVALID_ARG, "tune must be 0 or 1");
  if (o.store_bf16 != 0 && o.store_bf16 != 1) return fail(SIP_ERR_INVALID_ARG, "store_bf16 must be 0 or 1");
  if (o.store_bf16 && o.dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "store_bf16 needs SIP_F32");
  if (o.select_window != 0 && o.select_window != 1) return fail(SIP_ERR_INVALID_ARG, "select_window must be 0 or 1");
  return SIP_OK;
}

sip_status validate(const sip_grid *grid, const sip_set *sets, int nsets, const sip_options *opts) {
  sip_status st = check_grid(grid);
  if (st) return st;
  if (!sets) return fail(SIP_ERR_INVALID_ARG, "sets is NULL");
  if (!opts) return fail(SIP_ERR_INVALID_ARG, "opts is NULL");
  if (nsets < 1 || nsets > kMaxSets) return fail(SIP_ERR_INVALID_ARG, "nsets must be in [1, %d]", kMaxSets);
  const GridDesc g = grid_desc(*grid);
  int nblur = 0;
  for (int i = 0; i < nsets; ++i) {
    if ((st = check_set(g, sets[i], i))) return st;
    nblur += sets[i].op == SIP_OP_BLUR;
  }
  if (nblur > 1) return fail(SIP_ERR_INVALID_ARG, "at most one blur set per projection");
  if (opts->store_bf16)
    for (int i = 0; i < nsets; ++i)
      if (sets[i].op == SIP_OP_BLUR || sets[i].scope != SIP_SCOPE_ALL)
        return fail(SIP_ERR_INVALID_ARG, "store_bf16 is not available with blur or per-line sets");
  if (nblur && opts->levels > 1) return fail(SIP_ERR_INVALID_ARG, "a blur set runs on one level only");
  return check_opts(*opts);
}

void set_fastdiv(InstDev &d) {
  d.fz = make_fastdiv((uint32_t)d.nz);
  d.fx = make_fastdiv((uint32_t)d.nx);
  d.fzm = make_fastdiv((uint32_t)(d.nz > 1 ? d.nz - 1 : 1));
  d.fxm = make_fastdiv((uint32_t)(d.nx > 1 ? d.nx - 1 : 1));
}

// ----------------------------------------------------------------------------
// instance layout (host description; device pointers filled at placement)
// ----------------------------------------------------------------------------
InstLayout make_layout(const GridDesc &g, const sip_set *sets, int nsets, const sip_options &o) {
  InstLayout L;
  L.g = g;
  L.opts = o;
  InstDev &d = L.dev;
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
  d.p = nsets;
  d.alg1 = o.form == SIP_FORM_ALG1 ? 1 : 0;
  d.nb = nsets + d.alg1;
  d.hist = o.evol_hist;
  d.max_iter = o.max_iter;
  d.cg_iters = o.cg_iters;
  d.cg_max = o.cg_max;
  d.check_every = o.check_every;
  d.stop = o.stop;
  d.adapt = o.adapt;
  d.adapt_every = o.adapt_every;
  d.eps_feas = o.eps_feas;
  d.eps_evol = o.eps_evol;
  d.rho0 = o.rho0;
  d.gamma0 = o.gamma0;
  d.eps_corr = o.eps_corr;
  d.rho_ratio_max = o.rho_ratio_max;
  d.gamma_max = o.gamma_max;
  d.select_window = o.select_window;
  d.bf16 = o.store_bf16;
  // s^{k0} = A_i x^{k0} is recomputed from x^{k0}, which the x history ring
  // still holds when the adapt interval is shorter than the ring
  d.k0_ring = o.adapt_every < o.evol_hist ? 1 : 0;

  int64_t yoff = 0, woff = 0, soff = 0, boff = 0;
  int nseg = 0;
  L.blo.assign(d.nb, std::vector<double>());
  L.bhi.assign(d.nb, std::vector<double>());
  for (int b = 0; b < d.nb; ++b) {
    BlockDev &bd = d.blk[b];
    if (b < nsets) {
      const sip_set &s = sets[b];
      bd.op = s.op;
      const int t = s.type == SIP_SET_BOUNDS ? BT_BOUNDS
                    : s.type == SIP_SET_L1   ? BT_L1
                    : s.type == SIP_SET_L2   ? BT_L2
                    : s.type == SIP_SET_CARD ? BT_CARD
                                             : BT_ANNULUS;
      bd.type = (s.scope != SIP_SCOPE_ALL && t != BT_BOUNDS) ? BT_LINE : t;
      if (bd.type == BT_LINE) {
        bd.line_type = t;
        bd.scope = s.scope;
        int64_t dd[3];
        int stag;
        part_dims(g, op_parts(g, s.op)[0], dd, stag);
        const int a = s.scope - 1;  // axis of the lines
        bd.line_len = dd[a];
        bd.nlines = dd[0] * dd[1] * dd[2] / dd[a];
        bd.line_stride = a == 0 ? 1 : a == 1 ? dd[0] : dd[0] * dd[1];
        bd.line_a = a == 0 ? 1 : a == 1 ? dd[0] : dd[0] * dd[1];
        bd.line_b = a == 0 ? dd[0] : a == 1 ? dd[0] * dd[1] : 0;
      }
      bd.lo = s.lo;
      bd.hi = s.hi;
      bd.sigma_abs = s.sigma;
      bd.sigma_rel = (s.type == SIP_SET_L1 || s.type == SIP_SET_L2) ? s.sigma_rel : 0.0;
      bd.k_abs = s.k;
      bd.k_frac = s.type == SIP_SET_CARD ? s.k_frac : 0.0;
    } else {
      bd.op = SIP_OP_I;
      bd.type = BT_DIST;
    }
    bd.M = op_rows(g, bd.op);
    bd.yoff = yoff;
    yoff += bd.M;
    bd.bv_lo = bd.bv_hi = -1;
    if (b < nsets && sets[b].center_vec) {
      // l2 data fit: the observed values (NaN: unobserved) at bv_lo
      L.blo[b].assign(sets[b].center_vec, sets[b].center_vec + bd.M);
      bd.bv_lo = boff;
      boff += (bd.M + 3) / 4 * 4;
    }
    if (b < nsets && sets[b].op == SIP_OP_BLUR) {
      // the blur table: taps, autocorrelation, end correction (binary64)
      const sip_set &s = sets[b];
      const int R = s.blur_radius;
      auto k = [&](int t) { return t < 0 ? (-t <= R ? s.blur_taps[-t] : 0.0) : (t <= R ? s.blur_taps[t] : 0.0); };
      std::vector<double> &tb = L.blur;
      tb.assign(s.blur_taps, s.blur_taps + R + 1);
      for (int dd = 0; dd <= 2 * R; ++dd) {
        double a = 0.0;
        for (int t = -R; t <= R; ++t) a += k(t) * k(t + dd);
        tb.push_back(a);
      }
      for (int ii = 0; ii < R; ++ii)
        for (int l = 0; l < R; ++l) {
          double e = 0.0;
          for (int j = -R; j < 0; ++j) e += k(ii - j) * k(l - j);
          tb.push_back(e);
        }
      d.bl_R = R;
      d.bl_box = 1;
      for (int t = 1; t <= R; ++t) d.bl_box = d.bl_box && s.blur_taps[t] == s.blur_taps[0];
      d.bl_axis = s.blur_axis;
      d.bl_n = (int32_t)g.n[s.blur_axis];
      d.bl_blk = b;
      d.bl_st = s.blur_axis == 0 ? 1 : s.blur_axis == 1 ? g.n[0] : g.n[0] * g.n[1];
      d.bl_off = boff;
      boff += ((int64_t)tb.size() + 3) / 4 * 4;
      d.k0_ring = 0;  // s^{k0} = F x^{k0} is kept (k0s), not re-blurred from the ring
    }
    if (b < nsets && (sets[b].lo_vec || sets[b].hi_vec)) {
      const sip_set &s = sets[b];
      L.blo[b].resize(bd.M);
      L.bhi[b].resize(bd.M);
      for (int64_t j = 0; j < bd.M; ++j) {
        L.blo[b][j] = s.lo_vec ? s.lo_vec[j] : s.lo;
        L.bhi[b][j] = s.hi_vec ? s.hi_vec[j] : s.hi;
      }
      const int64_t Mp = (bd.M + 3) / 4 * 4;  // 16-byte aligned like y
      bd.bv_lo = boff;
      bd.bv_hi = boff + Mp;
      boff += 2 * Mp;
    }
    bd.woff = bd.soff = -1;
    bd.job_w = bd.job_s = -1;
    // w / s scratch regions start on 16-byte boundaries (vector loads)
    if (bd.type == BT_L1 || bd.type == BT_L2 || bd.type == BT_CARD || bd.type == BT_ANNULUS || bd.type == BT_LINE) {
      bd.woff = woff;
      woff += (bd.M + 3) / 4 * 4;
    }
    if (bd.type == BT_L1 || bd.type == BT_CARD || bd.type == BT_LINE) {
      bd.soff = soff;
      soff += (bd.M + 3) / 4 * 4;
    }
    bd.seg0 = nseg;
    int64_t row0 = 0;
    for (int kind : op_parts(g, bd.op)) {
      SegDev &sg = d.seg[nseg++];
      sg.kind = kind;
      sg.block = b;
      sg.row0 = row0;
      sg.len = part_rows(g, kind);
      row0 += sg.len;
    }
    bd.nseg = nseg - bd.seg0;
  }
  SegDev &ring = d.seg[nseg++];
  ring.kind = SEG_RING;
  ring.block = -1;
  ring.row0 = 0;
  ring.len = d.N;
  d.nseg = nseg;
  L.Mtot = yoff;
  L.Mw = woff;
  L.Ms = soff;
  L.Mb = boff;
  // selection jobs (local numbering; made global at placement)
  for (int b = 0; b < d.nb; ++b) {
    BlockDev &bd = d.blk[b];
    if (bd.type != BT_L1 && bd.type != BT_CARD) continue;
    for (int feas = 0; feas < 2; ++feas) {
      JobDev j;
      memset(&j, 0, sizeof j);
      j.block = b;
      j.kind = bd.type == BT_L1 ? JOB_L1 : JOB_TOPK;
      j.feas = feas;
      j.M = bd.M;
      j.data_off = feas ? bd.soff : bd.woff;
      j.ntiles = (int32_t)((bd.M + kTile - 1) / kTile);
      (feas ? bd.job_s : bd.job_w) = (int)L.jobs.size();
      L.jobs.push_back(j);
    }
  }
  return L;
}

// Algorithmic bytes per iteration of the fused schedule (see sip.h).
double layout_bytes_per_iter(const InstLayout &L, int dtype) {
  const InstDev &d = L.dev;
  const double W = (double)esize(dtype);
  const double N = (double)d.N, Mp = (double)L.Mtot;
  const int ncg = L.opts.cg_iters > 0 ? L.opts.cg_iters : 5;
  const int rsel = select_passes(dtype);
  double words = 2 * Mp + 2 * N + (d.alg1 ? 0 : N);  // rhs: y, v, x read; r write (+ m)
  // CG: w0 = C r0; per step p, x, r, w, s read and written, except in the
  // iteration's last step, after which only x is read again (r, p, x read,
  // x written)
  words += 3.0 * N + (ncg > 0 ? (ncg - 1) * 10.0 * N + 4.0 * N : 0.0);
  words += 4 * Mp + N + (d.alg1 ? N : 0);             // set pass: x, y, v read, y, v write (+ m)
  double feas = 0.0;
  for (int b = 0; b < d.nb; ++b) {
    const BlockDev &bd = d.blk[b];
    if (bd.type == BT_L2 || bd.type == BT_ANNULUS || bd.type == BT_LINE) words += 2.0 * bd.M;
    if (bd.type == BT_L1 || bd.type == BT_CARD) {
      words += (2.0 + rsel) * bd.M;
      feas += (1.0 + rsel) * bd.M;
    }
  }
  words += 2 * N;                                      // x history write + read
  if (L.opts.adapt && !L.opts.rho_schedule) words += 8 * Mp / L.opts.adapt_every;
  words += (feas + d.hist * N) / L.opts.check_every;
  return words * W;
}

// ----------------------------------------------------------------------------
// plan: one or more instances placed in one device arena
// ----------------------------------------------------------------------------
// One work item per CTA: `chunk` rows (a multiple of kTile) of one item.
static void push_tiles(std::vector<Tile> &v, int inst, int item, int64_t n, int64_t chunk) {
  int seq = 0;
  for (int64_t s = 0; s < n; s += chunk, ++seq) {
    Tile t;
    t.inst = inst;
    t.item = item;
    t.start = s;
    t.len = (int32_t)(n - s < chunk ? n - s : chunk);
    t.seq = seq;
    v.push_back(t);
  }
}

// Grid-point work items of an instance with a blur block: blocks of
// kBlurTZ z rows x kBlurTA samples along an x or y blur axis (item = kBlurTZ),
// or for a blur along z runs of one z column of at most kBlurLen samples
// (item = 1); start = the block's first grid point, len = item x samples.
static void push_blur_blocks(std::vector<Tile> &v, int inst, const InstDev &d) {
  int seq = 0;
  auto push = [&](int64_t g0, int tz, int ta) {
    Tile t;
    t.inst = inst;
    t.item = tz;
    t.start = g0;
    t.len = tz * ta;
    t.seq = seq++;
    v.push_back(t);
  };
  const int64_t nz = d.nz, nx = d.nx, ny = d.ny;
  if (d.bl_axis == 0) {
    const int64_t runs = (nz + kBlurLen - 1) / kBlurLen;
    const int ta = (int)((nz + runs - 1) / runs);
    for (int64_t col = 0; col < nx * ny; ++col)
      for (int64_t a0 = 0; a0 < nz; a0 += ta) push(a0 + nz * col, 1, ta);
    return;
  }
  const int64_t na = d.bl_axis == 1 ? nx : ny, no = d.bl_axis == 1 ? ny : nx;
  for (int64_t o = 0; o < no; ++o)
    for (int64_t a0 = 0; a0 < na; a0 += kBlurTA)
      for (int64_t z0 = 0; z0 < nz; z0 += kBlurTZ)
        push(z0 + nz * (d.bl_axis == 1 ? a0 + nx * o : o + nx * a0), kBlurTZ, kBlurTA);
}

// Rows per work item for a launch that covers `total` rows: `slots` CTAs
// (SMs x resident CTAs per SM, so the launch runs in one wave), a multiple
// of the CTA width, at most kMaxChunk.
static int64_t chunk_for(int64_t total, int64_t slots) {
  if (slots < 1) slots = 1;
  int64_t c = (total + slots - 1) / slots;
  c = (c + kThreads - 1) / kThreads * kThreads;
  if (c < kThreads) c = kThreads;
  if (c > kMaxChunk) c = kMaxChunk;
  return c;
}

// CTAs per cluster for instances of up to n grid points: about 8192 points
// per CTA, a power of two in [1, 16].
static int cluster_ctas_for(int64_t n) {
  int c = 1;
  while (c < 16 && (int64_t)c * 8192 < n) c *= 2;
  return c;
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return n > 0 ? n : 152;
}

void Plan::release() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  if (tgraph) cudaGraphExecDestroy(tgraph);
  tgraph = nullptr;
  if (d_ts) cudaFree(d_ts);
  d_ts = nullptr;
  tcat.clear();
  if (arena) cudaFree(arena);
  arena = nullptr;
}

static double clamp_scale(double v) { return v >= 1.0 / 16 && v <= 16.0 ? v : 1.0; }

void plan_tuning(const Plan &P, sip_tuning *out) { *out = P.knobs; }

sip_status plan_build(Plan &P, std::vector<InstLayout> &insts, int dtype, bool own_m, bool packed, bool dry,
                      const sip_tuning *tune) {
  P.dtype = dtype;
  P.ninst = (int)insts.size();
  const size_t W = esize(dtype);
  // ---- sizes
  int64_t njobs = 0, ntie = 0;
  std::vector<Tile> tn, trhs, tset, tsel, tfin, tline;
  P.any_card = P.any_fin = false;
  P.cg_launch = 0;
  P.max_iter = 0;
  P.check_every = 1 << 30;
  P.any_stop = false;
  // rows covered by each launch kind over all instances -> work-item size
  int64_t tot_n = 0, tot_set = 0, tot_fin = 0, tot_sel = 0, tot_line = 0;
  for (auto &L : insts) {
    tot_n += L.dev.N;
    for (int s = 0; s < L.dev.nseg; ++s) tot_set += L.dev.seg[s].len;
    for (int b = 0; b < L.dev.nb; ++b) {
      const int t = L.dev.blk[b].type;
      if (t == BT_L1 || t == BT_L2 || t == BT_CARD || t == BT_ANNULUS) tot_fin += L.dev.blk[b].M;
      if (t == BT_LINE) tot_line += L.dev.blk[b].nlines;
    }
    for (auto &j : L.jobs) tot_sel += j.M;
  }
  if (cudaError_t e = kernels_setup()) return fail(SIP_ERR_CUDA, "kernel set-up: %s", cudaGetErrorString(e));
  const int64_t sms = sm_count();
  // cluster execution: each instance's work items are sized for the CTAs of
  // one cluster (no blur blocks: their terms have no cluster-form bodies)
  bool any_blur0 = false;
  int64_t max_n = 0;
  for (auto &L : insts) {
    any_blur0 = any_blur0 || L.dev.bl_R != 0;
    if (L.dev.N > max_n) max_n = L.dev.N;
  }
  int exec_req = insts.empty() ? SIP_EXEC_GRAPH : insts[0].opts.exec;
  if (tune && (tune->exec == SIP_EXEC_GRAPH || tune->exec == SIP_EXEC_CLUSTER)) exec_req = tune->exec;
  const double sc_n = tune ? clamp_scale(tune->scale_n) : 1.0, sc_set = tune ? clamp_scale(tune->scale_set) : 1.0;
  const double sc_sel = tune ? clamp_scale(tune->scale_sel) : 1.0, sc_fin = tune ? clamp_scale(tune->scale_fin) : 1.0;
  auto slots = [&](int kind, double scale) {
    const double v = (double)sms * launch_occupancy(dtype, kind) * scale;
    return (int64_t)(v < 1.0 ? 1.0 : v);
  };
  P.cluster = 0;
  P.cluster_grid = 0;
  if (exec_req == SIP_EXEC_CLUSTER && !any_blur0) {
    int cs = (tune && tune->exec == SIP_EXEC_CLUSTER && tune->cluster_ctas > 0) ? tune->cluster_ctas
                                                                             : insts[0].opts.cluster_ctas;
    if (cs <= 0) cs = cluster_ctas_for(max_n);
    const int cap = fused_cluster_capacity(dtype, cs);
    if (cap > 0) {
      P.cluster = cs;
      P.cluster_grid = cap < P.ninst ? cap : P.ninst;
    }
  }
  const bool clustered = P.cluster > 0;
  const int64_t ch_n = chunk_for(tot_n, slots(0, sc_n));
  // Staged right-hand side for binary32 plans of 2D instances: the y / v
  // windows of a work item of ch rows take about 8 (rows + halo) bytes per
  // segment; the largest work item that lets 2 (else 1) CTAs share an SM.
  int64_t ch_rhs = 0;
  P.rhs_smem = 0;
  bool any_blur = false;
  for (auto &L : insts) any_blur = any_blur || L.dev.bl_R != 0;
  bool stageable = dtype == SIP_F32 && !insts.empty() && !any_blur && !clustered && !(tune && tune->stage_rhs == 0);
  for (auto &L : insts) stageable = stageable && L.dev.ny == 1 && L.dev.N < (int64_t(1) << 31);
  for (int occ = 2; stageable && occ >= 1 && !P.rhs_smem; --occ) {
    const int64_t ch = chunk_for(tot_n, (int64_t)((double)sms * occ * sc_n > 1.0 ? (double)sms * occ * sc_n : 1.0));
    size_t need = 0;
    for (auto &L : insts) {
      size_t b = 0;
      for (int sgi = 0; sgi < L.dev.nseg; ++sgi) {
        const int kind = L.dev.seg[sgi].kind;
        if (kind == SEG_RING) continue;
        const int64_t win = kind == SEG_DX ? ch + L.dev.nz : ch + 2;
        b += 2 * sizeof(float) * (size_t)(win + 8);
      }
      if (b > need) need = b;
    }
    if (need <= kRhsSmemMax && rhs_tma_occupancy(need) >= occ) {
      P.rhs_smem = need;
      ch_rhs = ch;
    }
  }
  const int64_t ch_set = chunk_for(tot_set, slots(1, sc_set));
  const int64_t ch_sel = chunk_for(tot_sel, slots(2, sc_sel));
  const int64_t ch_fin = chunk_for(tot_fin, slots(3, sc_fin));
  // per-line sets: one line per work item (a line's radix passes are short
  // and latency-bound; more CTAs in flight beat longer CTAs in one wave)
  const int64_t ch_line = 1;
  for (int i = 0; i < P.ninst; ++i) {
    InstLayout &L = insts[i];
    InstDev &d = L.dev;
    // work-item sizes: one wave of the whole GPU over all instances, or, in
    // cluster execution, this instance's rows over the cluster's CTAs
    int64_t ci_n = ch_n, ci_set = ch_set, ci_sel = ch_sel, ci_fin = ch_fin;
    if (clustered) {
      int64_t rows_set = 0, rows_fin = 0, rows_sel = 0;
      for (int sg = 0; sg < d.nseg; ++sg) rows_set += d.seg[sg].len;
      for (int b = 0; b < d.nb; ++b) {
        const int t = d.blk[b].type;
        if (t == BT_L1 || t == BT_L2 || t == BT_CARD || t == BT_ANNULUS) rows_fin += d.blk[b].M;
      }
      for (auto &j : L.jobs) rows_sel += j.M;
      ci_n = chunk_for(d.N, P.cluster);
      ci_set = chunk_for(rows_set, P.cluster);
      ci_sel = chunk_for(rows_sel, P.cluster);
      ci_fin = chunk_for(rows_fin, P.cluster);
    }
    if (tune && (tune->select_window == 0 || tune->select_window == 1)) d.select_window = tune->select_window;
    d.job0 = (int32_t)njobs;
    d.njob = (int32_t)L.jobs.size();
    for (int b = 0; b < d.nb; ++b) {
      if (d.blk[b].job_w >= 0) d.blk[b].job_w += (int32_t)njobs;
      if (d.blk[b].job_s >= 0) d.blk[b].job_s += (int32_t)njobs;
    }
    for (auto &j : L.jobs) {
      j.inst = i;
      j.hist_off = (int64_t)(njobs++) * kBins;
      // select passes walk the job in ch_sel items; tie counts follow the
      // final pass's ch_fin items of the job's block
      j.ntiles = (int32_t)((j.M + ci_sel - 1) / ci_sel);
      j.tie_off = ntie;
      ntie += (j.M + ci_fin - 1) / ci_fin;
    }
    const size_t b0 = tn.size();
    if (d.bl_R)
      push_blur_blocks(tn, i, d);
    else
      push_tiles(tn, i, 0, d.N, ci_n);
    d.nt_n = (int32_t)(tn.size() - b0);
    d.tn0 = (int32_t)b0;
    d.nt_rhs = 0;
    if (P.rhs_smem || any_blur) {
      // staged right-hand side items; in a plan with a blur block, the
      // right-hand side walks contiguous items (its blur part comes from
      // the block items' launch before it)
      const size_t br = trhs.size();
      push_tiles(trhs, i, 0, d.N, P.rhs_smem ? ch_rhs : ch_n);
      d.nt_rhs = (int32_t)(trhs.size() - br);
    }
    d.nt_part = d.nt_n > d.nt_rhs ? d.nt_n : d.nt_rhs;
    const size_t b1 = tset.size();
    for (int s = 0; s < d.nseg; ++s) push_tiles(tset, i, s, d.seg[s].len, ci_set);
    d.nt_set = (int32_t)(tset.size() - b1);
    d.tset0 = (int32_t)b1;
    const size_t b2 = tfin.size(), bl = tline.size();
    for (int b = 0; b < d.nb; ++b) {
      const int t = d.blk[b].type;
      if (t == BT_LINE) push_tiles(tline, i, b, d.blk[b].nlines, ch_line);
      if (t == BT_L1 || t == BT_L2 || t == BT_CARD || t == BT_ANNULUS) {
        push_tiles(tfin, i, b, d.blk[b].M, ci_fin);
        P.any_fin = true;
      }
      if (t == BT_CARD) P.any_card = true;
    }
    d.nt_fin = (int32_t)(tfin.size() - b2);
    d.tfin0 = (int32_t)b2;
    d.tline0 = (int32_t)bl;
    d.nt_line = (int32_t)(tline.size() - bl);
    const size_t bq = tsel.size();
    for (int j = 0; j < (int)L.jobs.size(); ++j) push_tiles(tsel, i, d.job0 + j, L.jobs[j].M, ci_sel);
    d.tsel0 = (int32_t)bq;
    d.nt_sel = (int32_t)(tsel.size() - bq);
    const int cgl = L.opts.cg_iters > 0 ? L.opts.cg_iters : L.opts.cg_max;
    if (cgl > P.cg_launch) P.cg_launch = cgl;
    if (L.opts.max_iter > P.max_iter) P.max_iter = L.opts.max_iter;
    if (L.opts.check_every < P.check_every) P.check_every = L.opts.check_every;
    if (L.opts.stop) P.any_stop = true;
  }
  // persistent execution needs every work list to fit the cooperative grid
  // in one pass per phase; otherwise (or on request) the graph path runs
  P.exec = insts.empty() ? SIP_EXEC_GRAPH : insts[0].opts.exec;
  P.fused_grid = fused_grid(dtype);
  // AUTO takes the graph path: measured on the 512 x 1024 five-set workload,
  // the persistent kernel (all phases in one register allocation, 2 CTAs
  // per SM) runs at half its speed
  if (P.exec == SIP_EXEC_AUTO) P.exec = SIP_EXEC_GRAPH;
  if (P.exec == SIP_EXEC_PERSISTENT && P.fused_grid <= 0) P.exec = SIP_EXEC_GRAPH;
  if (clustered)
    P.exec = SIP_EXEC_CLUSTER;
  else if (P.exec == SIP_EXEC_CLUSTER)
    P.exec = SIP_EXEC_GRAPH;
  if (tune && tune->exec == SIP_EXEC_GRAPH) P.exec = SIP_EXEC_GRAPH;
  // a blur block's terms live in their own instantiations of the
  // grid-point and set-pass kernels; the persistent kernel has none
  P.blur = false;
  P.blur_all = !insts.empty();
  for (auto &L : insts) {
    P.blur = P.blur || L.dev.bl_R != 0;
    P.blur_all = P.blur_all && L.dev.bl_R != 0;
  }
  if (P.blur) P.exec = SIP_EXEC_GRAPH;
  // the knobs this plan is built with
  memset(&P.knobs, 0, sizeof P.knobs);
  P.knobs.scale_n = sc_n;
  P.knobs.scale_set = sc_set;
  P.knobs.scale_sel = sc_sel;
  P.knobs.scale_fin = sc_fin;
  P.knobs.exec = P.exec;
  P.knobs.cluster_ctas = P.cluster;
  P.knobs.select_window = insts.empty() ? 1 : insts[0].dev.select_window;
  P.knobs.stage_rhs = P.rhs_smem ? 1 : 0;
  P.nt_n = (int)tn.size();
  P.nt_rhs = (int)trhs.size();
  P.nt_set = (int)tset.size();
  P.nt_sel = (int)tsel.size();
  P.nt_fin = (int)tfin.size();
  P.nt_line = (int)tline.size();
  P.njobs = (int)njobs;

  // ---- arena layout
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off = align_up(off + (bytes > 0 ? bytes : 0), 256);
    return o;
  };
  struct Offs {
    int64_t x, y, v, cr[2], cw[2], cs[2], cp, cgp, ring, w, s, k0s, k0vh, k0y, k0v, m, sched_r, sched_g, trace, bvec,
        bls;
  };
  std::vector<Offs> offs(P.ninst);
  // warm state (x, y, v) of all instances first, then the rest of the state,
  // then everything else: memsets stay contiguous
  // batched plans keep every instance's x (and m) back to back, so one copy
  // moves all outputs (inputs); instance i starts at element P.pack_off[i]
  P.pack_off.assign(P.ninst + 1, 0);
  for (int i = 0; i < P.ninst; ++i) P.pack_off[i + 1] = P.pack_off[i] + insts[i].dev.N;
  const int64_t o_xpack = packed ? take(P.pack_off[P.ninst] * W) : -1;
  for (int i = 0; i < P.ninst; ++i) {
    offs[i].x = packed ? o_xpack + P.pack_off[i] * W : take(insts[i].dev.N * W);
    offs[i].y = take(insts[i].Mtot * W);
    offs[i].v = take(insts[i].Mtot * W);
  }
  P.warm_end = off;
  for (int i = 0; i < P.ninst; ++i) {
    const InstLayout &L = insts[i];
    const int64_t N = L.dev.N;
    const bool ad = L.opts.adapt != 0;
    for (int j = 0; j < 2; ++j) {
      offs[i].cr[j] = take(N * W);
      offs[i].cw[j] = take(N * W);
      offs[i].cs[j] = take(N * W);
    }
    offs[i].cp = take(N * W);
    offs[i].cgp = take((int64_t)3 * 2 * L.dev.nt_part * W);  // accumulator type = storage type
    offs[i].ring = take((int64_t)L.dev.hist * N * W);
    offs[i].w = take(L.Mw * W);
    offs[i].s = take(L.Ms * W);
    offs[i].k0s = (ad && !L.dev.k0_ring) ? take(L.Mtot * W) : -1;
    offs[i].k0vh = ad ? take(L.Mtot * W) : -1;
    offs[i].k0y = ad ? take(L.Mtot * W) : -1;
    offs[i].k0v = ad ? take(L.Mtot * W) : -1;
  }
  P.state_end = off;
  const int64_t o_mpack = (own_m && packed) ? take(P.pack_off[P.ninst] * W) : -1;
  for (int i = 0; i < P.ninst; ++i) {
    const InstLayout &L = insts[i];
    offs[i].m = own_m ? (packed ? o_mpack + P.pack_off[i] * W : take(L.dev.N * W)) : -1;
    offs[i].sched_r = L.opts.rho_schedule ? take((int64_t)L.opts.max_iter * L.dev.nb * 8) : -1;
    offs[i].sched_g = L.opts.gamma_schedule ? take((int64_t)L.opts.max_iter * L.dev.nb * 8) : -1;
    offs[i].trace = L.opts.trace ? take((int64_t)L.opts.max_iter * (2 * L.dev.nb + 2 + L.dev.p) * 8) : -1;
    offs[i].bvec = L.Mb ? take(L.Mb * W) : -1;
    offs[i].bls = L.dev.bl_R ? take(L.dev.N * W) : -1;
  }
  const int64_t o_ctrl = take(8 * sizeof(uint32_t));  // grid barrier words + finished count
  const int64_t o_insts = take((int64_t)P.ninst * sizeof(InstDev));
  const int64_t o_scal = take((int64_t)P.ninst * sizeof(InstScal));
  const int64_t o_jobs = take((int64_t)njobs * sizeof(JobDev));
  const int64_t o_jscal = take((int64_t)njobs * sizeof(JobScal));
  P.hist_begin = off;
  // three histogram buffers per array: the selection passes rotate over them
  const int64_t o_hcnt = take(3 * (int64_t)njobs * kBins * 4);
  const int64_t o_hs1 = take(3 * (int64_t)njobs * kBins * 8);
  const int64_t o_hs2 = take(3 * (int64_t)njobs * kBins * 8);
  const int64_t o_hs3 = take(3 * (int64_t)njobs * kBins * 8);
  P.hist_end = off;
  const int64_t o_ties = take(ntie * 4);
  // window candidates (keys, W bytes each) of the top-k w-jobs
  int64_t ncand = 0;
  for (auto &L : insts)
    for (auto &j : L.jobs)
      if (j.kind == JOB_TOPK && !j.feas) ncand += kWinCap;
  const int64_t o_cand = take(ncand * W);
  const int64_t o_tn = take((int64_t)tn.size() * sizeof(Tile));
  const int64_t o_trhs = take((int64_t)trhs.size() * sizeof(Tile));
  const int64_t o_tset = take((int64_t)tset.size() * sizeof(Tile));
  const int64_t o_tsel = take((int64_t)tsel.size() * sizeof(Tile));
  const int64_t o_tfin = take((int64_t)tfin.size() * sizeof(Tile));
  const int64_t o_tline = take((int64_t)tline.size() * sizeof(Tile));
  P.arena_bytes = off;
  if (dry) return SIP_OK;  // size only (admission control)

  if (hook_alloc_fails() || cudaMalloc(&P.arena, (size_t)off) != cudaSuccess) {
    cudaGetLastError();
    P.arena = nullptr;
    return fail(SIP_ERR_OOM, "device allocation of %lld bytes failed", (long long)off);
  }
  char *base = (char *)P.arena;
  auto at = [&](int64_t o) -> void * { return o < 0 ? nullptr : (void *)(base + o); };
  P.h_insts.resize(P.ninst);
  P.layouts = insts;
  for (int i = 0; i < P.ninst; ++i) {
    InstDev &d = insts[i].dev;
    const Offs &o = offs[i];
    d.x = at(o.x);
    d.y = at(o.y);
    d.v = at(o.v);
    for (int j = 0; j < 2; ++j) {
      d.cr[j] = at(o.cr[j]);
      d.cw[j] = at(o.cw[j]);
      d.cs[j] = at(o.cs[j]);
    }
    d.cp = at(o.cp);
    d.cgp = at(o.cgp);
    d.ring = at(o.ring);
    d.w = at(o.w);
    d.s = at(o.s);
    d.k0s = at(o.k0s);
    d.k0vh = at(o.k0vh);
    d.k0y = at(o.k0y);
    d.k0v = at(o.k0v);
    d.m = at(o.m);
    d.rho_sched = (const double *)at(o.sched_r);
    d.gamma_sched = (const double *)at(o.sched_g);
    d.trace = (double *)at(o.trace);
    d.bvec = at(o.bvec);
    d.bl_w = d.bl_R ? (const char *)d.bvec + d.bl_off * W : nullptr;
    d.bl_s = at(o.bls);
    d.trace_w = 2 * d.nb + 2 + d.p;
    P.h_insts[i] = d;
    P.layouts[i] = insts[i];
  }
  // single instance: the CG launches take their work items and descriptor
  // fields as parameters (items of ch_n points from 0, as pushed above)
  memset(&P.cg_one, 0, sizeof P.cg_one);
  if (P.ninst == 1 && !P.blur) {  // a blur instance's items are blocks
    P.cg_one.d = cg_desc(P.h_insts[0]);
    P.cg_one.chunk = clustered ? chunk_for(P.h_insts[0].N, P.cluster) : ch_n;
    P.cg_one.on = 1;
  }
  P.m_own = own_m;
  P.packed = packed;
  P.x_pack = packed ? at(o_xpack) : nullptr;
  P.m_pack = (own_m && packed) ? at(o_mpack) : nullptr;
  P.d_ctrl = (uint32_t *)at(o_ctrl);
  for (int i = 0; i < P.ninst; ++i) {
    P.h_insts[i].ndone = P.d_ctrl + 4;
    insts[i].dev.ndone = P.d_ctrl + 4;
    P.layouts[i].dev.ndone = P.d_ctrl + 4;
    P.h_insts[i].err = insts[i].dev.err = P.layouts[i].dev.err = P.d_ctrl + 2;
  }
  P.d_insts = (InstDev *)at(o_insts);
  P.d_scal = (InstScal *)at(o_scal);
  P.d_jobs = (JobDev *)at(o_jobs);
  P.d_jscal = (JobScal *)at(o_jscal);
  P.d_hcnt = (uint32_t *)at(o_hcnt);
  P.d_hs1 = (double *)at(o_hs1);
  P.d_hs2 = (double *)at(o_hs2);
  P.d_hs3 = (double *)at(o_hs3);
  P.d_ties = (uint32_t *)at(o_ties);
  P.d_tn = (Tile *)at(o_tn);
  P.d_trhs = trhs.empty() ? nullptr : (Tile *)at(o_trhs);
  P.d_tset = (Tile *)at(o_tset);
  P.d_tsel = (Tile *)at(o_tsel);
  P.d_tfin = (Tile *)at(o_tfin);
  P.d_tline = tline.empty() ? nullptr : (Tile *)at(o_tline);

  std::vector<JobDev> jobs;
  int64_t cand_at = o_cand;
  for (auto &L : insts)
    for (auto &j : L.jobs) {
      jobs.push_back(j);
      if (j.kind == JOB_TOPK && !j.feas) {
        jobs.back().cand = at(cand_at);
        cand_at += (int64_t)kWinCap * W;
      }
    }
  CK(cudaMemset(P.arena, 0, (size_t)off));
  // per-entry bound vectors and blur tables, in the storage type
  for (int i = 0; i < P.ninst; ++i) {
    const InstLayout &L = insts[i];
    if (L.dev.bl_R) {
      char *dst = (char *)P.h_insts[i].bvec + L.dev.bl_off * W;
      if (dtype == SIP_F64) {
        CK(cudaMemcpy(dst, L.blur.data(), L.blur.size() * 8, cudaMemcpyHostToDevice));
      } else {
        std::vector<float> f(L.blur.begin(), L.blur.end());
        CK(cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    for (int b = 0; b < L.dev.nb; ++b) {
      const BlockDev &bd = L.dev.blk[b];
      if (bd.bv_lo < 0) continue;
      for (int side = 0; side < 2; ++side) {
        const std::vector<double> &src = side ? L.bhi[b] : L.blo[b];
        if (src.empty()) continue;  // a data-fit center has no upper vector
        char *dst = (char *)P.h_insts[i].bvec + (side ? bd.bv_hi : bd.bv_lo) * W;
        if (dtype == SIP_F64) {
          CK(cudaMemcpy(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice));
        } else {
          std::vector<float> f(src.begin(), src.end());
          CK(cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
        }
      }
    }
  }
  // single instance with its own model copy: the descriptor (now complete,
  // the same bytes as its device copy) is immutable, so every kernel takes
  // it as a launch parameter
  memset(&P.one, 0, sizeof P.one);
  if (P.ninst == 1 && own_m) {
    P.one.d = P.h_insts[0];
    P.one.on = 1;
  }
  CK(cudaMemcpy(P.d_insts, P.h_insts.data(), P.ninst * sizeof(InstDev), cudaMemcpyHostToDevice));
  if (njobs) CK(cudaMemcpy(P.d_jobs, jobs.data(), njobs * sizeof(JobDev), cudaMemcpyHostToDevice));
  if (!tn.empty()) CK(cudaMemcpy(P.d_tn, tn.data(), tn.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  if (!trhs.empty()) CK(cudaMemcpy(P.d_trhs, trhs.data(), trhs.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  if (!tset.empty()) CK(cudaMemcpy(P.d_tset, tset.data(), tset.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  if (!tsel.empty()) CK(cudaMemcpy(P.d_tsel, tsel.data(), tsel.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  if (!tfin.empty()) CK(cudaMemcpy(P.d_tfin, tfin.data(), tfin.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  if (!tline.empty()) CK(cudaMemcpy(P.d_tline, tline.data(), tline.size() * sizeof(Tile), cudaMemcpyHostToDevice));
  return SIP_OK;
}

int64_t plan_bytes(const std::vector<InstLayout> &insts, int dtype, bool own_m, bool packed) {
  Plan P;
  std::vector<InstLayout> copy = insts;
  if (plan_build(P, copy, dtype, own_m, packed, true) != SIP_OK) return -1;
  return P.arena_bytes;
}

// ----------------------------------------------------------------------------
// launch sequencing
// ----------------------------------------------------------------------------
// Launches of one iteration.
static int launches_per_iter(const Plan &P) {
  return 3 + P.cg_launch + (P.nt_sel ? select_passes(P.dtype) : 0) + (P.any_card ? 1 : 0) + (P.nt_line ? 1 : 0) +
         (P.nt_fin ? 1 : 0) + 1 + (P.blur ? 2 : 0) + (P.blur && !P.blur_all ? P.cg_launch : 0);
}

// marks: every launch stamps its own slot pair of P.d_ts (timing graph)
static sip_status enqueue_iteration(Plan &P, cudaStream_t st, bool marks) {
  Launch L{P.dtype, st};
  L.blur = P.blur;
  auto T0 = [&](int c) {
    if (!marks) return;
    L.ts = P.d_ts + 2 * P.tcat.size();
    P.tcat.push_back(c);
  };
  auto T1 = [&](int) {};
  T0(KT_RHS);
  if (P.rhs_smem) {
    CK(launch_rhs_tma(L, P.d_trhs, P.nt_rhs, P.d_insts, P.d_scal, P.rhs_smem, P.one));
  } else if (P.blur) {
    CK(launch_blur_rhs(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal));
    T0(KT_RHS);
    CK(launch_rhs(L, P.d_trhs, P.nt_rhs, P.d_insts, P.d_scal, P.one));
  } else {
    CK(launch_rhs(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal, P.one));
  }
  T1(KT_RHS);
  T0(KT_CG_W0);
  CK(launch_cg_w0(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal, P.cg_one));  // w_0 = C r_0
  T1(KT_CG_W0);
  for (int j = 0; j < P.cg_launch; ++j) {
    if (j == P.cg_launch - 1 && !P.blur) {  // the iteration's last step: x only
      T0(KT_CG_LAST);
      CK(launch_cg_last(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal, 2 + j, P.cg_one));
      T1(KT_CG_LAST);
      break;
    }
    T0(KT_CG_STEP);
    if (!P.blur_all)
      CK(launch_cg_step(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal, 2 + j, P.cg_one));  // one CG step
    if (P.blur) {  // the blur instances' block items
      if (!P.blur_all) T0(KT_CG_STEP);
      CK(launch_cg_step_blur(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal, 2 + j));
    }
    T1(KT_CG_STEP);
  }
  if (P.blur) {  // s = F x of the blur blocks, read by the set pass
    T0(KT_SETPASS);
    CK(launch_blur_fwd(L, P.d_tn, P.nt_n, P.d_insts, P.d_scal));
    T1(KT_SETPASS);
  }
  T0(KT_SETPASS);
  CK(launch_setpass(L, P.d_tset, P.nt_set, P.d_insts, P.d_scal, P.d_jscal, P.d_jobs, P.one));
  T1(KT_SETPASS);
  if (P.nt_sel) {
    const int np = select_passes(P.dtype);
    for (int pass = 0; pass < np; ++pass) {
      T0(KT_SELECT);
      CK(launch_select(L, P.d_tsel, P.nt_sel, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_hcnt, P.d_hs1, P.d_hs2,
                       P.d_hs3, (int64_t)P.njobs * kBins, pass, P.one));
      T1(KT_SELECT);
    }
  }
  if (P.any_card) {
    T0(KT_TIES);
    CK(launch_ties(L, P.d_tfin, P.nt_fin, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_ties, P.one));
    T1(KT_TIES);
  }
  if (P.nt_line) {
    T0(KT_FINAL);  // per-line sets
    CK(launch_lines(L, P.d_tline, P.nt_line, P.d_insts, P.d_scal, P.one));
    T1(KT_FINAL);
  }
  if (P.nt_fin) {
    T0(KT_FINAL);
    CK(launch_final(L, P.d_tfin, P.nt_fin, P.d_insts, P.d_scal, P.d_jobs, P.d_jscal, P.d_ties, P.one));
    T1(KT_FINAL);
  }
  T0(KT_TAIL);
  CK(launch_tail(L, P.d_insts, P.d_scal, P.d_jscal, P.ninst, P.cg_launch, P.one));
  T1(KT_TAIL);
  return SIP_OK;
}

static sip_status capture(Plan &P, cudaStream_t cap, int iters, bool marks, cudaGraphExec_t *out) {
  CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  sip_status st = SIP_OK;
  for (int i = 0; i < iters && st == SIP_OK; ++i) st = enqueue_iteration(P, cap, marks);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(SIP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(SIP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return SIP_OK;
}

static sip_status build_graph(Plan &P, cudaStream_t cap, int iters) {
  if (P.graph && P.graph_iters == iters) return SIP_OK;
  if (P.graph) {
    cudaGraphExecDestroy(P.graph);
    P.graph = nullptr;
  }
  sip_status s = capture(P, cap, iters, false, &P.graph);
  if (!s) P.graph_iters = iters;
  return s;
}

static sip_status build_timing_graph(Plan &P, cudaStream_t cap, int iters) {
  if (P.tgraph && P.tgraph_iters == iters) return SIP_OK;
  if (P.tgraph) cudaGraphExecDestroy(P.tgraph);
  P.tgraph = nullptr;
  if (P.d_ts) cudaFree(P.d_ts);
  P.d_ts = nullptr;
  P.tcat.clear();
  const size_t words = 2 * (size_t)launches_per_iter(P) * iters;
  if (cudaMalloc(&P.d_ts, words * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    P.d_ts = nullptr;
    return fail(SIP_ERR_OOM, "timing stamps: device allocation failed");
  }
  sip_status s = capture(P, cap, iters, true, &P.tgraph);
  if (!s && 2 * P.tcat.size() > words) return fail(SIP_ERR_INTERNAL, "timing stamps: launch count");
  if (!s) P.tgraph_iters = iters;
  return s;
}

// Run `iters` iterations (kernels no-op once an instance is done).
static sip_status run_persistent(Plan &P, cudaStream_t st, int iters) {
  FusedLaunch F;
  F.tn = P.d_tn;
  F.tset = P.d_tset;
  F.tsel = P.d_tsel;
  F.tfin = P.d_tfin;
  F.tline = P.d_tline;
  F.nt_line = P.nt_line;
  F.nt_n = P.nt_n;
  F.nt_set = P.nt_set;
  F.nt_sel = P.nt_sel;
  F.nt_fin = P.nt_fin;
  F.insts = P.d_insts;
  F.scal = P.d_scal;
  F.jobs = P.d_jobs;
  F.jscal = P.d_jscal;
  F.hcnt = P.d_hcnt;
  F.hs1 = P.d_hs1;
  F.hs2 = P.d_hs2;
  F.hs3 = P.d_hs3;
  F.hstride = (int64_t)P.njobs * kBins;
  F.ties = P.d_ties;
  F.bar = P.d_ctrl;
  F.ndone = P.d_ctrl + 4;
  F.ninst = P.ninst;
  F.cg_launch = P.cg_launch;
  F.any_card = P.any_card ? 1 : 0;
  F.any_fin = P.any_fin ? 1 : 0;
  F.iters = iters;
  F.bar_extra = g_hooks.bar_extra;
  F.bar_spins = g_hooks.bar_spins;
  CK(launch_fused(Launch{P.dtype, st}, F, P.fused_grid));
  return SIP_OK;
}

// Cluster form: one launch runs every iteration; each instance stops on its
// own (max_iter or the stopping rule), so the host polls nothing.
static sip_status run_cluster(Plan &P, cudaStream_t st, int iters) {
  FusedLaunch F;
  memset(&F, 0, sizeof F);
  F.tn = P.d_tn;
  F.tset = P.d_tset;
  F.tsel = P.d_tsel;
  F.tfin = P.d_tfin;
  F.tline = P.d_tline;
  F.nt_line = P.nt_line;
  F.nt_n = P.nt_n;
  F.nt_set = P.nt_set;
  F.nt_sel = P.nt_sel;
  F.nt_fin = P.nt_fin;
  F.insts = P.d_insts;
  F.scal = P.d_scal;
  F.jobs = P.d_jobs;
  F.jscal = P.d_jscal;
  F.hcnt = P.d_hcnt;
  F.hs1 = P.d_hs1;
  F.hs2 = P.d_hs2;
  F.hs3 = P.d_hs3;
  F.hstride = (int64_t)P.njobs * kBins;
  F.ties = P.d_ties;
  F.bar = P.d_ctrl;
  F.ndone = P.d_ctrl + 4;
  F.ninst = P.ninst;
  F.cg_launch = P.cg_launch;
  F.any_card = P.any_card ? 1 : 0;
  F.any_fin = P.any_fin ? 1 : 0;
  F.iters = iters;
  CK(launch_fused_cluster(Launch{P.dtype, st}, F, P.cluster_grid, P.cluster));
  return SIP_OK;
}

sip_status run_iterations(Plan &P, cudaStream_t st, cudaStream_t cap, int iters, bool poll, int32_t *pinned_flag,
                          KernelTimer *tm) {
  const NvtxRange range("sip: iterations");
  if (!tm && P.exec == SIP_EXEC_PERSISTENT) return run_persistent(P, st, iters);
  if (!tm && P.exec == SIP_EXEC_CLUSTER) return run_cluster(P, st, iters);
  const int chunk = poll ? P.check_every : (iters < 10 ? iters : 10);
  if (tm) {
    // per-kernel device time: the stamping graph, its stamps read after each replay
    sip_status s = build_timing_graph(P, cap, chunk);
    if (s) return s;
    std::vector<unsigned long long> ts(2 * P.tcat.size());
    for (int done_iters = 0; done_iters < iters;) {
      CK(cudaMemsetAsync(P.d_ts, 0xff, ts.size() * sizeof(unsigned long long), st));
      CK(cudaGraphLaunch(P.tgraph, st));
      done_iters += chunk;
      CK(cudaMemcpyAsync(ts.data(), P.d_ts, ts.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (size_t i = 0; i < P.tcat.size(); ++i) {
        const unsigned long long t0 = ts[2 * i], t1 = ~ts[2 * i + 1];
        tm->ms[P.tcat[i]] += t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
        tm->launches[P.tcat[i]] += 1;
      }
      if (poll && done_iters < iters) {
        CK(cudaMemcpyAsync(pinned_flag, P.d_ctrl + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*pinned_flag >= P.ninst) break;
      }
    }
    return SIP_OK;
  }
  sip_status s = build_graph(P, cap, chunk);
  if (s) return s;
  int done_iters = 0;
  while (done_iters < iters) {
    CK(cudaGraphLaunch(P.graph, st));
    done_iters += chunk;
    if (poll && done_iters < iters) {
      // every instance done?  (the tails count finished instances)
      CK(cudaMemcpyAsync(pinned_flag, P.d_ctrl + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*pinned_flag >= P.ninst) break;
    }
  }
  return SIP_OK;
}

sip_status plan_prepare(Plan &P, cudaStream_t st, bool warm) {
  const NvtxRange range(warm ? "sip: prepare (warm state)" : "sip: prepare");
  const Launch L{P.dtype, st};
  char *base = (char *)P.arena;
  if (warm) {
    CK(cudaMemsetAsync(base + P.warm_end, 0, (size_t)(P.state_end - P.warm_end), st));
    for (int i = 0; i < P.ninst; ++i)  // x^0 into the history ring
      CK(cudaMemcpyAsync(P.h_insts[i].ring, P.h_insts[i].x, (size_t)P.h_insts[i].N * esize(P.dtype),
                         cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemsetAsync(base, 0, (size_t)P.state_end, st));
  }
  CK(cudaMemsetAsync(base + P.hist_begin, 0, (size_t)(P.hist_end - P.hist_begin), st));
  CK(cudaMemsetAsync(P.d_ctrl, 0, 8 * sizeof(uint32_t), st));
  CK(launch_init(L, P.d_insts, P.d_scal, P.d_jscal, P.ninst));
  CK(launch_norms(L, P.d_tset, P.nt_set, P.d_insts, P.d_scal));
  return SIP_OK;
}

sip_status plan_set_m(Plan &P, int inst, const void *m, cudaStream_t st) {
  if (P.m_own && !P.packed) {
    // the plan's own copy: the descriptor (a launch parameter of the
    // captured graphs) stays valid for every model
    CK(cudaMemcpyAsync((void *)P.h_insts[inst].m, m, (size_t)P.h_insts[inst].N * esize(P.dtype),
                       cudaMemcpyDeviceToDevice, st));
    return SIP_OK;
  }
  P.h_insts[inst].m = m;
  CK(cudaMemcpyAsync(&P.d_insts[inst].m, &P.h_insts[inst].m, sizeof(void *), cudaMemcpyHostToDevice, st));
  return SIP_OK;
}

}  // namespace sip
