// Host-side launchers of the library's kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdlib>

#include "common.cuh"

namespace cl {

// Scheduling priority of an op's launches.  With the two-stream
// factorisation the panel chain (stream 0) runs at the device's highest
// priority and the bulk updates (stream 1) at its lowest; the priority is
// given as a launch attribute, which stream capture records in the graph's
// kernel nodes (a stream's own priority does not carry into a graph).
constexpr int kNoPrio = 0x7fffffff;
inline int op_priority(const Plan& p, const Op& op) {
  return p.streams[1] ? (op.stream ? p.prio_lo : p.prio_hi) : kNoPrio;
}
// Programmatic dependent launch of the front kernels (each opens with
// pdl_enter): on unless CLSELINV_PDL=0.
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("CLSELINV_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}
// launch options of one kernel: priority, and whether it may start launching
// while its predecessor in the stream still runs (only where that
// predecessor is a kernel of the same op list and no event wait lies between)
struct LaunchOpt {
  int prio = kNoPrio;
  bool pdl = false;
};
inline LaunchOpt op_launch(const Plan& p, const Op& op) { return {op_priority(p, op), op.pdl && pdl_enabled()}; }
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, LaunchOpt o,
                     Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2]{};
  unsigned n = 0;
  if (o.prio != kNoPrio) {
    attr[n].id = cudaLaunchAttributePriority;
    attr[n].val.priority = o.prio;
    ++n;
  }
  if (o.pdl) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cfg.attrs = n ? attr : nullptr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// one scheduled operation of the factorisation / selected inversion
template <typename T, typename R>
cudaError_t launch_op(const Plan& p, const Op& op, T* arena, const double* links, double m, double mu,
                      double* Gdiag, double* Gfwd, double* Gbwd, cudaStream_t st);

// batched complex GEMM over the descriptors of one OP_GEMM
cudaError_t launch_gemm(const Plan& p, const Op& op, double2* arena, cudaStream_t st);
cudaError_t launch_gemm(const Plan& p, const Op& op, float2* arena, cudaStream_t st);
// FP64-accurate GEMM on the BF16 tensor cores (split pass + digit GEMM)
cudaError_t launch_gemm_emu(const Plan& p, const Op& op, double2* arena, cudaStream_t st);
cudaError_t emu_prepare();
cudaError_t panel_prepare();
// split pass + tcgen05 digit GEMM over descriptors [d0, d1) with ndig digits
// per operand (3, 7 or 8); blocks = output
// tiles (128 x 16 complex); persistent kernels (single_chunk: every K <= 32)
// on min(blocks, max_ctas) CTAs, each a contiguous range of tiles
cudaError_t launch_emu(const GemmDesc* gd, const EmuDesc* ed, int d0, int d1, int items, int blocks, int batch,
                       double2* arena, int64_t stride, unsigned* words, int* ints, int64_t wstride, int64_t istride,
                       int* status, bool single_chunk, int max_ctas, int ndig, cudaStream_t st, LaunchOpt lo,
                       unsigned long long wait_ns);

// stochastic estimator (stochastic.cu): row-vector solves w = eta^dag D^{-1}
// with the factors in the fronts, in a workspace of stochastic_work_elems
// complex elements, and the estimated selected blocks
int64_t stochastic_work_elems(const Plan& p, int n);
template <typename T>
cudaError_t launch_left_solve(const Plan& p, const double* eta, int n, double* w, double2* work, cudaStream_t st);
cudaError_t launch_stoch_blocks(const Plan& p, const double* eta, const double* w, int n, double* Gd, double* Gf,
                                double* Gb, cudaStream_t st);

// fermion drift of every link of every replica
cudaError_t launch_drift(const Plan& p, const double* links, const double* Gfwd, const double* Gbwd, double mu,
                         double nf, double* Kf, cudaStream_t st);

// ---- Langevin step (langevin.cu) ----
// scalar arguments of the update / step-size rule
struct LangevinArgs {
  double eps_max, kappa;  // eps = min(eps_max, kappa / K_max), kappa <= 0: eps_max
  double fixed_eps;       // > 0: use this step and `step` instead of the rule and the state
  unsigned long long seed;
  long long step;
  int renorm_det = 0;     // 1: U <- U / det(U)^{1/3} after the update
  int reunit = 0;         // 1: U projected onto SU(3) after the update (Gram-Schmidt rows)
};
// observables record per replica (doubles): plaq_s re,im | plaq_t re,im | poly re,im |
// poly_inv re,im | condensate re,im | unitarity | K_max | eps | t | step | spare |
// density re,im | spare, spare
constexpr int kObsFields = 20;
// Langevin state per replica (doubles): t | step | eps of the last step | spare
constexpr int kStateFields = 4;

cudaError_t launch_gauge_drift(const Plan& p, const double* U, double* Ui, double beta, double* K, int acc,
                               cudaStream_t st);
cudaError_t launch_kmax(const Plan& p, const double* K, unsigned long long* slots, cudaStream_t st);
cudaError_t launch_update(const Plan& p, double* U, const double* K, const LangevinArgs& a,
                          const unsigned long long* slots, const double* state, cudaStream_t st);
cudaError_t launch_cool(const Plan& p, double* U, int n_cool, double alpha0, double* F, double* Om, double* Omi,
                        unsigned long long* slots, cudaStream_t st);
cudaError_t launch_obs_partial(const Plan& p, const double* U, double* Ui, const double* Gdiag, const double* Gfwd,
                               const double* Gbwd, double mu, double* part, bool invert, cudaStream_t st);
cudaError_t launch_obs_final(const Plan& p, const double* part, bool has_g, double nf, const unsigned long long* slots,
                             const LangevinArgs& a, double* state, double* obs, int advance, cudaStream_t st);
int obs_partial_doubles(const Plan& p);

}  // namespace cl
