// Host-side launchers of the device kernels (internal to libsip.so).
#pragma once

#include <cuda_runtime.h>

#include "sip_dev.cuh"

namespace sip {

struct Launch {
  int dtype;  // SIP_F64 / SIP_F32
  cudaStream_t stream;
  // launch-time stamps (timing runs only): [0] earliest CTA start, [1]
  // latest CTA end, global timer nanoseconds; null otherwise
  unsigned long long *ts = nullptr;
  // the plan has a blur block: the right-hand side, CG and set-pass
  // launches take the instantiations with the F^T F and F terms
  bool blur = false;
};

// iteration kernels (kernels.cu)
cudaError_t launch_init(const Launch &L, const InstDev *insts, InstScal *scal, JobScal *jscal, int ninst);
cudaError_t launch_norms(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal);
cudaError_t launch_rhs(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, const InstOne &one);
// staged right-hand side (binary32, 2D instances): `smem` bytes of y / v
// windows per CTA, at most kRhsSmemMax
constexpr size_t kRhsSmemMax = 200 * 1024;
cudaError_t launch_rhs_tma(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                           size_t smem, const InstOne &one);
int rhs_tma_occupancy(size_t smem);
cudaError_t launch_cg_w0(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const CgOne &one);
// ph: 2 for the first step launch of an iteration, then 3, 4, ...
cudaError_t launch_cg_step(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, int ph,
                           const CgOne &one);
// the last step launch of an iteration: x_{i+1} only (plans without a blur block)
cudaError_t launch_cg_last(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, int ph,
                           const CgOne &one);
// the blur block's right-hand side part F^T (rho y + v) - rho F^T F x, and
// s = F x, at the blur instances' block work items (plans with a blur block)
cudaError_t launch_cg_step_blur(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                                int ph);
cudaError_t launch_blur_rhs(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, const InstScal *scal);
cudaError_t launch_blur_fwd(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, const InstScal *scal);
cudaError_t launch_setpass(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                           JobScal *jscal, const JobDev *jobs, const InstOne &one);
// hstride: elements between the three histogram buffers the passes rotate
// over, or 0 for a single buffer
cudaError_t launch_select(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                          const JobDev *jobs, JobScal *jscal, uint32_t *hcnt, double *hs1, double *hs2, double *hs3,
                          int64_t hstride, int pass, const InstOne &one);
// BF16 storage trial: n binary32 values rounded in place to bfloat16
cudaError_t launch_round_bf16(const Launch &L, void *a, int64_t n);
// warm-start penalties of instance 0 (one value per block)
struct Penalties {
  double rho[kMaxBlocks], gamma[kMaxBlocks];
};
cudaError_t launch_load_penalties(cudaStream_t st, const InstDev *insts, InstScal *scal, const Penalties &pen);
// kernel attribute set-up, done once per device with that device current
// (call outside stream capture); devices 0..kMaxDevices-1
constexpr int kMaxDevices = 64;
cudaError_t kernels_setup();
// CTAs per SM for the kernels of a work-item list: 0 grid points, 1 set
// segments, 2 selection jobs, 3 final-pass blocks
int launch_occupancy(int dtype, int kind);
int select_passes(int dtype);

// persistent cooperative form of the iteration (kernels.cu)
struct FusedLaunch {
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
  uint32_t *bar;          // 4 words: arrivals, generation, error, unused
  const uint32_t *ndone;  // finished instances
  int ninst, cg_launch, any_card, any_fin, iters;
  uint32_t bar_extra;     // arrivals beyond the grid a barrier waits for (test hook; 0)
  long long bar_spins;    // polls before a barrier gives up (0: the default)
};
cudaError_t launch_fused(const Launch &L, const FusedLaunch &F, int grid);
int fused_grid(int dtype);
// cluster form: `clusters` clusters of `csize` CTAs, each running whole
// instances (all iterations) with the cluster barrier between phases
cudaError_t launch_fused_cluster(const Launch &L, const FusedLaunch &F, int clusters, int csize);
// clusters of csize CTAs of the cluster kernel resident at once (0: none fits)
int fused_cluster_capacity(int dtype, int csize);
cudaError_t launch_ties(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                        const JobDev *jobs, JobScal *jscal, uint32_t *ties, const InstOne &one);
// Per-line sets: one CTA per work item of lines (item = block, start/len =
// lines), after the set pass.
cudaError_t launch_lines(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal, const InstOne &one);
// Parallel Dykstra: x = mean_i y_i, v_i = x + v_i - y_i (p blocks of n packed).
cudaError_t launch_dykstra_update(const Launch &L, const void *y, void *v, void *x, int p, int64_t n);
cudaError_t launch_final(const Launch &L, const Tile *tiles, int nt, const InstDev *insts, InstScal *scal,
                         const JobDev *jobs, const JobScal *jscal, const uint32_t *ties, const InstOne &one);
// cg_launch: step launches per iteration
cudaError_t launch_tail(const Launch &L, const InstDev *insts, InstScal *scal, JobScal *jscal, int ninst,
                        int cg_launch, const InstOne &one);

// single-step operators on one grid (kernels.cu): `in` describes the grid and
// the segments of one operator; `sc` carries the stencil coefficients.
cudaError_t launch_apply_op(const Launch &L, const InstDev *in, const void *x, void *s, int64_t rows);
cudaError_t launch_apply_op_t(const Launch &L, const InstDev *in, const void *s, void *x, int64_t n);
cudaError_t launch_system_apply(const Launch &L, const InstDev *in, const InstScal *sc, const void *x, void *out,
                                int64_t n);

// multilevel transfer (kernels_ml.cu); dims are (nz, nx, ny) of the arrays
cudaError_t launch_restrict(const Launch &L, const int64_t fine[3], const int64_t coarse[3], const void *mf, void *mc);
cudaError_t launch_prolong(const Launch &L, const int64_t cdims[3], const int64_t fdims[3], int stagger_axis,
                           const void *uc, void *uf);

}  // namespace sip
