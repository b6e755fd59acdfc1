// Host-side plan / handle structures of libsip.so (internal).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "sip.h"
#include "sip_dev.cuh"

namespace sip {

// A named NVTX range for the lifetime of the object: the host phases of a
// projection (preparation, iteration replays, multilevel transfers) show as
// ranges in a timeline profiler; without one attached the calls are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

extern thread_local std::string g_err;
sip_status fail(sip_status s, const char *fmt, ...);

// Host-side fault injection for the failure-handling tests (sip_test_hook).
struct TestHooks {
  int fail_alloc = 0;          // the n-th next arena allocation fails (0: off)
  uint32_t bar_extra = 0;      // extra arrivals the persistent kernel's barriers wait for
  long long bar_spins = 0;     // polls before a barrier gives up (0: default)
};
extern TestHooks g_hooks;
// true when the hook says this arena allocation must fail
bool hook_alloc_fails();

struct GridDesc {
  int ndim;
  int64_t n[3];
  double h[3];
  int64_t N() const { return n[0] * n[1] * n[2]; }
};

struct InstLayout {
  GridDesc g;
  sip_options opts;
  InstDev dev;
  int64_t Mtot = 0, Mw = 0, Ms = 0;
  int64_t Mb = 0;  // per-entry bound vectors (lo and hi of every such block)
  std::vector<std::vector<double>> blo, bhi;  // per block, empty for scalar bounds
  std::vector<double> blur;                   // blur table of the blur block (empty: none)
  std::vector<JobDev> jobs;
};

// kernel categories of the per-kernel timer
enum KernelCat { KT_RHS = 0, KT_CG_W0, KT_CG_STEP, KT_SETPASS, KT_SELECT, KT_TIES, KT_FINAL, KT_TAIL, KT_CG_LAST, KT_COUNT };

// Per-kernel device time by category (opt-in): the iterations run as a CUDA
// graph whose kernels stamp their first CTA start and last CTA end with the
// global timer; the stamps are read after each replay.
struct KernelTimer {
  double ms[KT_COUNT] = {};
  int64_t launches[KT_COUNT] = {};
  void reset() {
    for (int c = 0; c < KT_COUNT; ++c) {
      ms[c] = 0.0;
      launches[c] = 0;
    }
  }
};

struct Plan {
  int dtype = SIP_F32;
  int ninst = 0;
  void *arena = nullptr;
  int64_t arena_bytes = 0;
  int64_t warm_end = 0, state_end = 0, hist_begin = 0, hist_end = 0;
  bool m_own = false;
  InstDev *d_insts = nullptr;
  InstScal *d_scal = nullptr;
  JobDev *d_jobs = nullptr;
  JobScal *d_jscal = nullptr;
  uint32_t *d_hcnt = nullptr;
  double *d_hs1 = nullptr, *d_hs2 = nullptr, *d_hs3 = nullptr;
  uint32_t *d_ties = nullptr;
  Tile *d_tn = nullptr, *d_tset = nullptr, *d_tsel = nullptr, *d_tfin = nullptr, *d_tline = nullptr;
  int nt_n = 0, nt_set = 0, nt_sel = 0, nt_fin = 0, nt_line = 0, njobs = 0;
  // staged right-hand side: its own work items and shared-memory bytes (0: not staged)
  Tile *d_trhs = nullptr;
  int nt_rhs = 0;
  size_t rhs_smem = 0;
  bool any_card = false, any_fin = false, any_stop = false;
  bool blur = false;      // an instance has a blur block (graph path, blur kernels)
  bool blur_all = false;  // every instance has one (no general CG step launches)
  CgOne cg_one;  // CG launch parameters of a single-instance plan (on = 0 otherwise)
  InstOne one;   // the descriptor as a launch parameter (single instance owning its model)
  int cg_launch = 0, max_iter = 0, check_every = 1;
  std::vector<InstDev> h_insts;
  std::vector<InstLayout> layouts;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  // timing graph: the same iterations, every launch stamping its slot pair
  cudaGraphExec_t tgraph = nullptr;
  int tgraph_iters = 0;
  unsigned long long *d_ts = nullptr;  // 2 words per launch of the timing graph
  std::vector<int> tcat;               // kernel category of launch i
  uint32_t *d_ctrl = nullptr;  // grid-barrier words [0..3], finished-instance count [4]
  bool packed = false;         // batched plan: x (and m) of all instances back to back
  std::vector<int64_t> pack_off;
  void *x_pack = nullptr, *m_pack = nullptr;
  int exec = SIP_EXEC_GRAPH;
  int fused_grid = 0;
  sip_tuning knobs;      // the launch-shape knobs it was built with
  int cluster = 0;       // CTAs per cluster in cluster execution (0: not clustered)
  int cluster_grid = 0;  // clusters launched: min(instances, clusters resident at once)
  void release();
};

GridDesc grid_desc(const sip_grid &g);
std::vector<int> op_parts(const GridDesc &g, int op);
int64_t part_rows(const GridDesc &g, int kind);
int64_t op_rows(const GridDesc &g, int op);
void part_dims(const GridDesc &g, int kind, int64_t d[3], int &stag);
sip_status validate(const sip_grid *grid, const sip_set *sets, int nsets, const sip_options *opts);
void set_fastdiv(InstDev &d);
InstLayout make_layout(const GridDesc &g, const sip_set *sets, int nsets, const sip_options &o);
double layout_bytes_per_iter(const InstLayout &L, int dtype);
// The plan's launch-shape knobs (sip_tuning): null = the heuristic.
sip_status plan_build(Plan &P, std::vector<InstLayout> &insts, int dtype, bool own_m, bool packed = false,
                      bool dry = false, const sip_tuning *tune = nullptr);
// the knobs a plan was built with (the heuristic's values when untuned)
void plan_tuning(const Plan &P, sip_tuning *out);
// device bytes plan_build would allocate for these instances (no allocation)
int64_t plan_bytes(const std::vector<InstLayout> &insts, int dtype, bool own_m, bool packed);
sip_status plan_prepare(Plan &P, cudaStream_t st, bool warm);
sip_status plan_set_m(Plan &P, int inst, const void *m, cudaStream_t st);
sip_status run_iterations(Plan &P, cudaStream_t st, cudaStream_t cap, int iters, bool poll, int32_t *pinned_flag,
                          KernelTimer *tm);

}  // namespace sip
