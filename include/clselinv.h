/*
 * clselinv.h -- C ABI of the GB300 selected-inversion fermion drift library.
 *
 * Bloch & Schenk, "Selected inversion as key to a stable Langevin evolution
 * across the QCD phase boundary" (arXiv:1707.08874).
 *
 * The library computes, for the staggered Dirac matrix D(m;mu) of Eq. 1 on an
 * Ns^3 x Nt torus with SL(3,C) links, the 3x3 blocks of D^{-1} on the pattern
 * of D (Sec. 3, the "selected inversion": a sparse LU followed by a backward
 * sweep that never forms an inverse entry outside the filled pattern) and from
 * them the fermion drift K^f of Eq. 6, written as Tr(P B) + Tr(Q F) (Eq. 8).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) doubles ("complex128").
 *  - Site index s = ((t*Ns + z)*Ns + y)*Ns + x, V = Ns^3 Nt; direction
 *    nu = 0..3 is x, y, z, t; colour indices a, b = 0..2.
 *  - links  [B][V][4][3][3]: U_{s,nu}, row a, column b.
 *  - D_{s,s} = m; D_{s,s+nu} = +1/2 eta_nu(s) s_nu(s) e^{+mu d_{nu,t}} U_{s,nu};
 *    D_{s+nu,s} = -1/2 eta_nu(s) s_nu(s) e^{-mu d_{nu,t}} U_{s,nu}^{-1}, with
 *    eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z) and
 *    s_nu(s) = -1 on temporal hops between t = Nt-1 and t = 0 (antiperiodic),
 *    else +1.  U^{-1} replaces U^dagger so that SL(3,C) links are allowed.
 *  - Every pointer argument named as a device array is a caller-owned,
 *    contiguous device pointer (cudaMalloc / torch tensor data_ptr()).  The
 *    library never frees or retains caller memory.
 *  - Every compute call is stream-ordered on the given stream (NULL = legacy
 *    default stream), allocates nothing and does not synchronise the host.
 *  - Return values are CL_* status codes.  Launch-time failures come back
 *    directly; numerical failures (a tiny pivot, a non-finite result) are
 *    recorded in a device status word and read with cl_get_status().
 *
 * Environment (tuning only; results are bitwise the same either way)
 * ------------------------------------------------------------------
 *  - CLSELINV_CHAIN_SMS=n: SMs the bulk digit-GEMM launches of a two-stream
 *    factorisation leave free for the panel chain (default 2; read when a
 *    plan is created).
 *  - CLSELINV_PDL=0: no programmatic dependent launch between the front
 *    kernels (default on; read once per process).
 *  - CLSELINV_FOLD_GROUPS=2: two instead of four fold groups in the
 *    persistent digit GEMM (read once per process).
 *
 * Environment (precision; changes results within the precision's accuracy)
 * --------------------------------------------------------------------------
 *  - CLSELINV_EMU_DIGITS=7: CL_FP64_EMU plans created afterwards split their
 *    GEMM operands into 7 instead of 8 base-256 digits (an FP64 GEMM's
 *    accuracy instead of ~2^-58 of the row / column maxima; fewer tensor-core
 *    products), for accuracy and speed comparisons.
 */
#ifndef CLSELINV_H
#define CLSELINV_H

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CL_OK 0
#define CL_ERR_INVALID_ARG 1
#define CL_ERR_OOM 2
#define CL_ERR_CUDA 3
#define CL_ERR_SINGULAR 4
#define CL_ERR_NONFINITE 5
#define CL_ERR_TIMEOUT 6
#define CL_ERR_UNSUPPORTED 7

/* arithmetic of the sparse factorisation and selected inversion */
#define CL_FP64 0       /* all front arithmetic in FP64 (FP64 tensor-core MMA) */
#define CL_MIXED_FP32 1 /* FP32 fronts, FP64 input/output and drift            */
#define CL_FP64_EMU 2   /* FP64 fronts; the front GEMMs run as 8-digit BF16
                           products on the tensor cores, accurate to ~2^-58 of
                           the operands' row / column maxima (below the FP64
                           rounding of the result)                              */
#define CL_MIXED_BF16X3 3 /* the mixed form: FP64 fronts, FP64 pivot-block
                           (panel) inverses with partial pivoting; Schur-
                           complement updates and off-diagonal selected-inverse
                           GEMMs as split-BF16x3 products (3 digits, FP32
                           accumulation, FP32-class accuracy); the panel
                           products with the pivot-block inverse and the
                           diagonal blocks G_JJ of the selected-inverse sweep
                           with 7 digits (FP64 accuracy)                        */

typedef struct cl_plan cl_plan;
typedef struct cl_group cl_group;

/* Summary of a plan (host values, no device access). */
typedef struct cl_plan_info {
  int Ns, Nt, V, N;          /* lattice and matrix order N = 3V (ragged plan:
                                Ns = Nt = 0, V = sites of all its lattices)    */
  int batch;                 /* replicas per call (ragged: lattices per call)   */
  int precision;             /* CL_FP64, CL_MIXED_FP32, CL_FP64_EMU or CL_MIXED_BF16X3 */
  int n_supernodes;          /* separators of the nested dissection            */
  int n_levels;              /* height of the elimination tree + 1              */
  int max_front;             /* largest front order (unknowns)                  */
  int max_pivot_block;       /* largest supernode (pivot unknowns)              */
  int panel;                 /* pivoting panel width (unknowns, multiple of 3)  */
  double factor_flops;       /* real flops of one factorisation (per replica;
                                ragged: averaged over its lattices)            */
  double selinv_flops;       /* real flops of one selected inversion (same)     */
  double front_bytes;        /* device bytes of the front pool (all replicas)   */
  double device_bytes;       /* all device memory held by the plan              */
  int launches_per_eval;     /* library kernel launches of one cl_drift_eval    */
  double workspace_bytes;    /* digit workspace of CL_FP64_EMU / CL_MIXED_BF16X3 (all replicas) */
  int n_shapes;              /* lattice shapes: 1, or nshapes of cl_analyze_ragged */
} cl_plan_info;

/* Per-kernel timing record filled by cl_profile_read. */
typedef struct cl_profile_entry {
  char name[32];             /* kernel family: "gemm", "panel_inverse", ...     */
  int launches;              /* launches recorded since cl_profile_enable       */
  double total_ms;           /* sum of CUDA-event durations of those launches   */
  double flops;              /* algorithmic real flops of those launches        */
  double bytes;              /* algorithmic DRAM bytes of those launches        */
} cl_profile_entry;

/* One launch of a profiled call, filled by cl_profile_trace. */
typedef struct cl_trace_entry {
  char name[32];             /* kernel family, as in cl_profile_entry           */
  int phase;                 /* 0 factorisation op, 1 selected-inversion op, -1 other */
  int op;                    /* index of the op in its phase's list (-1 other)   */
  int stream;                /* factorisation stream: 0 panel chain, 1 bulk     */
  int level;                 /* tree level of the op (root = highest; -1 none)  */
  double t0_us, t1_us;       /* event times around the launch, microseconds from
                                the first recorded launch                       */
} cl_trace_entry;

/* Parameters of one complex-Langevin step (cl_langevin_step). */
typedef struct cl_langevin_params {
  double beta;               /* Wilson coupling: S_g = beta sum_P [1 - (Tr U_P + Tr U_P^{-1})/6] */
  double m, mu;              /* quark mass and chemical potential of D(m;mu)   */
  double nf;                 /* factor of the fermion drift (1 = unrooted det D) */
  double eps_max;            /* largest Langevin step                           */
  double kappa;              /* adaptive step eps = min(eps_max, kappa/K_max);
                                kappa <= 0 keeps eps = eps_max                  */
  double alpha_cool;         /* gauge-cooling step alpha0 (alpha = alpha0 / max_x |f_x|) */
  unsigned long long seed;   /* key of the Philox4x32-10 noise stream           */
  int n_cool;                /* gauge-cooling iterations after each update     */
  int fermions;              /* 1: K = K^g + K^f (selected inversion); 0: K^g only */
  int renorm_det;            /* 1: after each update U <- U / det(U)^{1/3} (principal cube
                                root), removing the drift of det U away from 1; 0: off
                                (default, as in the paper: Sec. 4.2 keeps the links free
                                rather than reunitarising, for consistency with mu != 0) */
  int reunit;                /* 1: after each update (and determinant renormalisation) every
                                link is projected onto SU(3): first row normalised, second
                                row orthogonalised to it and normalised, third row the
                                complex conjugate of their cross product -- the
                                reunitarisation Sec. 4.2 names as the remedy of the wrong
                                mu = 0 results (there the evolution should stay in SU(3));
                                0: off (default, as in the paper's runs)              */
} cl_langevin_params;

/*
 * Record layouts used by the Langevin calls (device arrays of doubles):
 *   state [B][4]:  t (Langevin time) | step count | eps of the last step | spare
 *                  (caller zero-initialises; the step count keys the noise)
 *   obs   [B][20]: plaq_s re,im | plaq_t re,im | P re,im | P' re,im |
 *                  condensate re,im | unitarity norm | K_max | eps | t | step | spare |
 *                  density re,im | spare, spare
 *   plaquettes (1/3) Tr U_P averaged over the 3V spatial / 3V temporal
 *   plaquettes; P, P' = (1/(3 Ns^3)) sum Tr prod_t U_{x,t}^{+1 / -1};
 *   condensate = (nf/V) sum_x Tr G_xx; unitarity = (1/4V) sum Tr(U U^dag) - 3;
 *   density n = (nf/V) Tr(G dD/dmu) = (nf/V) d log det D / d mu, from the
 *   temporal blocks G_{x,x+t}, G_{x+t,x} only (Sec. 3: the fermionic
 *   observables need only G where D is non-zero).
 */

/*
 * cl_analyze -- symbolic analysis, done once per lattice shape (Sec. 3: the
 * "sparse LU" needs an ordering; the paper's solver does not describe its
 * own, this library uses geometric nested dissection of the 4D torus).
 *   Ns, Nt     even extents >= 4 (even for the staggered phases, >= 4 so that
 *              s+nu and s-nu are distinct sites)
 *   batch      number of independent lattices (replicas) per call, >= 1
 *   precision  CL_FP64, CL_MIXED_FP32, CL_FP64_EMU or CL_MIXED_BF16X3
 *   plan       out: library-owned handle, release with cl_destroy_plan
 * Builds the elimination tree, supernodes, front index maps and the launch
 * schedule on the host, then allocates and uploads all device memory the
 * later calls need on the current device.  Returns CL_ERR_INVALID_ARG for bad
 * extents, CL_ERR_OOM / CL_ERR_CUDA on allocation or copy failure.
 */
int cl_analyze(int Ns, int Nt, int batch, int precision, cl_plan** plan);

/*
 * cl_analyze_ex -- cl_analyze with an explicit pivoting-panel width
 * (unknowns, a multiple of 3 in 3..48; 0 = the precision's default: 48 for
 * CL_FP64, 30 for the other precisions).  Narrower panels shorten the
 * serial chain of FP64 panel inverses, wider ones make fewer, larger GEMMs;
 * the autotuner in the Python package picks it per shape by timing.
 */
int cl_analyze_ex(int Ns, int Nt, int batch, int precision, int panel, cl_plan** plan);

/*
 * cl_analyze_ragged -- one plan over lattices of several shapes (Sec. 4: the
 * paper's runs span lattice sizes; production batches mix them):
 *   nshapes     number of shapes, >= 1
 *   Ns, Nt      host arrays [nshapes]: extents of each shape (even, >= 4)
 *   count       host array [nshapes]: lattices (replicas) of each shape, >= 1
 *   precision   as cl_analyze
 *   plan        out: library-owned handle, release with cl_destroy_plan
 * Every shape is analysed once; the fronts of all lattices of all shapes lie
 * side by side in one arena and one fixed schedule runs them level by level
 * (height above the leaves), so each step of every level -- panel inverses,
 * tensor-core GEMMs over all their output tiles, copies, extend-adds and
 * gathers -- is one launch across all shapes and replicas; persistent GEMM
 * CTAs take tile ranges of that launch regardless of the lattice they belong
 * to.  The per-site steps (assembly, extraction, drift) run one launch per
 * shape.  The compute calls cl_factor, cl_selinv_blocks, cl_fermion_drift and
 * cl_drift_eval take the site-indexed arrays of all lattices concatenated in
 * shape order, each shape's replicas in order: links [sum_i count_i V_i][4][3][3],
 * Gdiag [..][3][3], Gfwd / Gbwd [..][4][3][3], Kf [..][4][8], V_i = Ns_i^3 Nt_i.
 * The Langevin calls return CL_ERR_UNSUPPORTED on a ragged plan, and
 * cl_plan_get_node too.  Returns CL_ERR_INVALID_ARG for bad shapes or counts
 * (more than 65535 lattices), CL_ERR_OOM / CL_ERR_CUDA on allocation failure.
 */
int cl_analyze_ragged(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, cl_plan** plan);
/* cl_analyze_ragged_ex -- cl_analyze_ragged with an explicit pivoting-panel
 * width, common to all shapes (as cl_analyze_ex). */
int cl_analyze_ragged_ex(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, int panel,
                         cl_plan** plan);

/*
 * cl_analyze_symbolic -- the host half of cl_analyze only (no device memory,
 * usable without a GPU).  The plan supports cl_plan_get_info and
 * cl_plan_get_node; compute calls on it return CL_ERR_INVALID_ARG.
 */
int cl_analyze_symbolic(int Ns, int Nt, int precision, cl_plan** plan);
/* cl_analyze_symbolic_ex -- the same with an explicit pivot-panel width (as cl_analyze_ex). */
int cl_analyze_symbolic_ex(int Ns, int Nt, int precision, int panel, cl_plan** plan);
/* cl_analyze_ragged_symbolic -- the host half of cl_analyze_ragged_ex (panel
 * 0 = the precision's default); supports the plan queries and exports. */
int cl_analyze_ragged_symbolic(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, int panel,
                               cl_plan** plan);

/*
 * cl_factor -- numeric sparse LU of D(m;mu) (Sec. 3, first half of the
 * selected inversion), multifrontal, for every replica.
 *   links   device [B][V][4][3][3] complex128, read only
 *   m, mu   quark mass and chemical potential
 * Pivoting is partial pivoting restricted to diagonal panels of at most
 * info.panel unknowns inside each supernode; a panel pivot below
 * 1e-13 * max|panel| records CL_ERR_SINGULAR in the status word.
 */
int cl_factor(cl_plan* plan, const double* links, double m, double mu, cudaStream_t stream);

/*
 * cl_selinv_blocks -- backward (Takahashi) sweep of the selected inversion
 * from the root to the leaves, then extraction of the blocks of G = D^{-1}
 * where D is non-zero (Sec. 3, Eq. 8).  Requires a preceding cl_factor.
 *   Gdiag  device out [B][V][3][3]     G_{s,s}
 *   Gfwd   device out [B][V][4][3][3]  G_{s,s+nu}   (the block P of Eq. 8)
 *   Gbwd   device out [B][V][4][3][3]  G_{s+nu,s}   (the block Q of Eq. 8)
 * Any output pointer may be NULL to skip it.
 */
int cl_selinv_blocks(cl_plan* plan, double* Gdiag, double* Gfwd, double* Gbwd,
                     cudaStream_t stream);

/*
 * cl_fermion_drift -- Eq. 6 through Eq. 8 for every link:
 *   K^f_{a,s,nu} = nf * [Tr(G_{s,s+nu} B_a) + Tr(G_{s+nu,s} F_a)],
 *   F_a = d_a D_{s,s+nu}, B_a = d_a D_{s+nu,s}, d_a U = i lambda_a U
 *   (left Lie derivative, Gell-Mann lambda_a in the standard order).
 *   links      device [B][V][4][3][3]
 *   Gfwd/Gbwd  device [B][V][4][3][3] from cl_selinv_blocks
 *   mu         chemical potential used in cl_factor
 *   nf         overall factor (1.0 = the unrooted det D of Eq. 1)
 *   Kf         device out [B][V][4][8] complex128
 * Non-finite results record CL_ERR_NONFINITE in the status word.
 */
int cl_fermion_drift(cl_plan* plan, const double* links, const double* Gfwd, const double* Gbwd,
                     double mu, double nf, double* Kf, cudaStream_t stream);

/*
 * cl_drift_eval -- cl_factor + cl_selinv_blocks + cl_fermion_drift in one
 * call (one "fermion-drift evaluation").  Gdiag may be NULL; Gfwd, Gbwd and
 * Kf are required.
 */
int cl_drift_eval(cl_plan* plan, const double* links, double m, double mu, double nf,
                  double* Gdiag, double* Gfwd, double* Gbwd, double* Kf, cudaStream_t stream);

/*
 * Stochastic estimator of the fermion drift (Sec. 3, Eq. 7), the comparison
 * path the paper contrasts with the exact drift:
 *   tr[D^{-1} d_{axnu} D] ~ (1/n) sum_i eta_i^dag D^{-1} (d_{axnu} D) eta_i,
 * for noise vectors with E[eta eta^dag] = 1 (Z2, Z4, U(1) or Gaussian entries).
 * Site-indexed noise arrays hold every lattice of the plan: eta, w
 * [n][sites][3] complex, sites = batch x V (single shape, replicas in order) or
 * the sites of all lattices of a ragged plan (in the plan's order).
 *
 * cl_stochastic_workspace -- bytes of device workspace the calls below need
 *   for n noise vectors (two front-vector sets per noise vector and replica).
 *
 * cl_left_solve -- w_i = eta_i^dag D^{-1} (row vectors, w_i[z] the entries of
 *   eta_i^dag D^{-1} at site z) from the factors of the preceding cl_factor:
 *   forward over the elimination tree (leaves to root) r_S <- r_S - r_J U-hat,
 *   backward (root to leaves) w_J = r_J A_JJ^{-1} + w_S (-L-hat), with the
 *   front blocks A_JJ^{-1}, U-hat = A_JJ^{-1} A_JS, L-hat = A_SJ A_JJ^{-1}
 *   left by cl_factor.  Must run before cl_selinv_blocks, which overwrites
 *   the factors.
 *   eta   device [n][sites][3], read only;  n in 1..65535
 *   w     device out [n][sites][3]
 *   work  device scratch of cl_stochastic_workspace bytes (16-byte aligned),
 *         caller-owned, not used by another call in flight
 *
 * cl_stochastic_drift -- cl_factor + cl_left_solve + the estimated selected
 *   blocks Gfwd_est[x][nu] = (1/n) sum_i eta_i[x] w_i[x+nu]^T, Gbwd_est[x][nu] =
 *   (1/n) sum_i eta_i[x+nu] w_i[x]^T, Gdiag_est[x] = (1/n) sum_i eta_i[x] w_i[x]^T
 *   (expectations: the exact blocks G_{x,x+nu}, G_{x+nu,x}, G_{x,x}) + the
 *   drift of Eq. 8 from them, which is the estimator above link by link.
 *   links, m, mu, nf, Kf as cl_drift_eval; Gdiag_est may be NULL.
 */
int cl_stochastic_workspace(const cl_plan* plan, int n, size_t* bytes);
int cl_left_solve(cl_plan* plan, const double* eta, int n, double* w, void* work, size_t work_bytes,
                  cudaStream_t stream);
int cl_stochastic_drift(cl_plan* plan, const double* links, double m, double mu, double nf, const double* eta, int n,
                        double* w, double* Gdiag_est, double* Gfwd_est, double* Gbwd_est, double* Kf, void* work,
                        size_t work_bytes, cudaStream_t stream);

/*
 * cl_gauge_drift -- gauge part of Eq. 5 for the Wilson action:
 *   K^g_{a,s,nu} = (i beta/6) sum_{6 staples A} Tr[lambda_a (U A - A^{-1} U^{-1})]
 *   (A the staple with Tr U_P = Tr(U_{s,nu} A)), i.e. K^g = -d_a S_g.
 *   links device [B][V][4][3][3]; Kg device out [B][V][4][8].
 */
int cl_gauge_drift(cl_plan* plan, const double* links, double beta, double* Kg, cudaStream_t stream);

/*
 * cl_link_update -- Eq. 3-4 with a fixed step: U <- R U,
 *   R = exp(i sum_a lambda_a (eps K_a + sqrt(eps) eta_a)),
 * eta_a real Gaussian, <eta_a eta_b> = 2 delta_ab, from Philox4x32-10 with
 * counter (4 s + nu, half, step, replica) and key = seed, Box-Muller on
 * u = (x + 1/2) 2^-32 (half 0 gives eta_1..4, half 1 eta_5..8).
 *   links device in/out [B][V][4][3][3]; K device [B][V][4][8]; eps > 0.
 */
int cl_link_update(cl_plan* plan, double* links, const double* K, double eps, unsigned long long seed,
                   long long step, cudaStream_t stream);

/*
 * cl_gauge_cool -- n_cool steepest-descent steps of gauge cooling (Sec. 4.1
 * names it; the form follows the unitarity-norm gradient):
 *   f_x = sum_nu [U_{x,nu} U_{x,nu}^dag - U_{x-nu,nu}^dag U_{x-nu,nu}] (traceless),
 *   alpha = alpha0 / max_x |f_x|_F, Omega_x = exp(-alpha f_x),
 *   U_{x,nu} <- Omega_x U_{x,nu} Omega_{x+nu}^{-1}.
 */
int cl_gauge_cool(cl_plan* plan, double* links, int n_cool, double alpha0, cudaStream_t stream);

/*
 * cl_observables -- plaquettes, Polyakov loops, unitarity norm, and from the
 * selected blocks (when given) the chiral condensate (Gdiag) and the quark-
 * number density (Gfwd, Gbwd at chemical potential mu), into obs [B][20]
 * (layout above; eps, t, step fields are zero).  Gdiag/Gfwd/Gbwd may be NULL.
 */
int cl_observables(cl_plan* plan, const double* links, const double* Gdiag, const double* Gfwd, const double* Gbwd,
                   double mu, double nf, double* obs, cudaStream_t stream);

/*
 * cl_langevin_step -- one stochastic Euler step of Eq. 3-5 for every replica:
 * drift K = K^g + K^f (K^f by the selected inversion of D(m;mu)), adaptive
 * step eps = min(eps_max, kappa / K_max), observables of the configuration
 * before the update (condensate from this step's G_xx), the update with noise
 * keyed by (seed, state.step), n_cool gauge-cooling steps, then
 * state.t += eps, state.step += 1.
 *   links device in/out; prm host struct; state device [B][4]; obs device [B][20].
 */
int cl_langevin_step(cl_plan* plan, double* links, const cl_langevin_params* prm, double* state, double* obs,
                     cudaStream_t stream);

/*
 * cl_drift_eval_noalloc -- the same evaluation as cl_drift_eval (FP64 fronts on
 * the FP64 tensor pipe, one lattice) for callers that cannot allocate device
 * memory where they need a drift: host runtimes whose device memory belongs to
 * another allocator (a framework's caching allocator that has reserved the
 * GPU), plugins that must not grow the process's footprint per call, loops
 * that cannot afford the device-wide synchronisation cudaMalloc / cudaFree may
 * cause.  The paper has no counterpart; this is a deployment convenience.
 *   Ns, Nt         lattice; fronts + workspace + tables must fit the fixed
 *                  20 MiB device scratch array (4^4, V = 256, fits; larger
 *                  shapes return CL_ERR_UNSUPPORTED before any device work)
 *   links, m, mu, nf, Gdiag (may be NULL), Gfwd, Gbwd, Kf: as cl_drift_eval,
 *                  caller-owned device arrays for one lattice (batch 1)
 * Allocates no device memory: the scratch is a file-scope device array that
 * every GPU loading the library holds until the process exits.  Set-up work
 * happens on first use: the first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and caches it, and the first call for
 * a lattice shape on a device analyses the shape on the host and uploads its
 * index tables into the array (synchronising the stream once); later calls
 * with the same shape reuse them and issue only a clear of the status word
 * and the kernels.  Make these first calls before any stream capture.  The
 * cached address does not survive cudaDeviceReset: do not call the entry
 * point again in a process after it.  All calls share the one array, which
 * keeps the last call's contents (the fronts are cleared by the evaluation
 * itself): calls that overlap on the GPU (different streams, or different
 * host threads) race and corrupt each other.  Numerical status (singular
 * pivot, non-finite drift) is not reported; check the outputs.
 */
int cl_drift_eval_noalloc(int Ns, int Nt, const double* links, double m, double mu, double nf,
                          double* Gdiag, double* Gfwd, double* Gbwd, double* Kf, cudaStream_t stream);

/*
 * cl_zgemm_emu -- FP64-accurate complex GEMM on the BF16 tensor cores, the
 * kernel behind CL_FP64_EMU (the dense front products of Sec. 3 - Schur
 * updates and selected-inverse blocks - as one call):
 *   C = [C if beta] + (-1 if neg) * A B
 *   M, N, K     >= 1
 *   A           device, M x K complex (interleaved re, im doubles), row-major, lda >= K
 *   B           device, K x N complex, row-major, ldb >= N
 *   C           device, M x N complex, row-major, ldc >= N (in / out); must not overlap A or B
 *   beta, neg   0 or 1
 *   work        device scratch of cl_zgemm_emu_workspace bytes, 256-byte aligned,
 *               caller-owned, not used by another call in flight
 *   status      device int[4] (caller-owned, zeroed by the caller): a tensor-core
 *               wait that gives up records CL_ERR_TIMEOUT in status[0]
 * A, B, C must be 16-byte aligned.  Each operand element is split into seven
 * 8-bit digits per row (A) / column (B) and per 32-element k chunk; the 28
 * leading digit products run as BF16 tcgen05 MMAs with FP32 accumulators in
 * tensor memory, folded in triple-float and rounded once to FP64.  The paper
 * computes in FP64; this path reproduces an FP64 GEMM's accuracy.  Returns
 * CL_ERR_INVALID_ARG for bad sizes, strides, alignment or a short workspace,
 * CL_ERR_CUDA on a launch failure; stream-ordered, no host synchronisation.
 */
int cl_zgemm_emu_workspace(int M, int N, int K, size_t* bytes);
int cl_zgemm_emu(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                 int beta, int neg, void* work, size_t work_bytes, int* status, cudaStream_t stream);

/*
 * cl_get_status -- synchronises `stream`, returns the first numerical error
 * recorded since the last call (CL_OK if none) in *info and clears it.
 * detail (may be NULL) receives the supernode and panel column of a
 * singular pivot, or -1.
 */
int cl_get_status(cl_plan* plan, cudaStream_t stream, int* info, int* detail);

/*
 * cl_plan_pivot_growth -- synchronises `stream` and returns in *growth the
 * largest pivot growth of the latest factorisation's panel blocks:
 * max |entry| / min |pivot| of each Gauss-Jordan block (magnitudes as
 * max(|re|, |im|); +inf for a zero pivot; 0 before any factorisation).
 * Pivots are chosen among the rows of a panel and of the next panel of its
 * supernode (static across supernodes, Sec. 3); a large growth means an
 * ill-conditioned pivot block that amplifies the rounding of everything
 * updated through it (on 8^3x4 lattices, m = 0.05, mu = 0.25: growths of
 * 11-62 over twenty configurations, errors of the FP64 path <= 2e-11; with
 * pivots restricted to each panel the growth reached ~1e3 and the error
 * 1.6e-9).  Reset by every factorisation (cl_factor, cl_drift_eval); not
 * cleared by cl_get_status.  CL_ERR_INVALID_ARG for a symbolic plan or a
 * null pointer.
 */
int cl_plan_pivot_growth(cl_plan* plan, cudaStream_t stream, double* growth);

/*
 * cl_plan_set_wait_limit -- limit of the waits of the tensor-core GEMM roles
 * (producer, MMA issuer, fold warps) for a later launch of this plan's
 * compute calls: seconds in [0, 0.5]; a negative value restores the default
 * 0.5 s.  A wait that runs out records CL_ERR_TIMEOUT in the status word;
 * the kernel then waits (with the full 0.5 s bound) for the copies and MMAs it
 * has in flight, frees its tensor memory and returns, and the results of
 * that evaluation are undefined.  Not part of the paper: it lets a test run
 * the timeout path (a limit of 0 gives up at the first unfinished wait)
 * without a kernel that never signals.
 */
int cl_plan_set_wait_limit(cl_plan* plan, double seconds);

/* cl_plan_get_info -- host summary of a plan. */
int cl_plan_get_info(const cl_plan* plan, cl_plan_info* info);

/*
 * cl_plan_get_node -- the structure of supernode i (0 <= i < n_supernodes,
 * postorder: children before parents, the root last).
 *   parent     out: parent supernode or -1
 *   level      out: height above the leaves (0 = leaf)
 *   n_sep      out: number of sites eliminated at this supernode
 *   n_bnd      out: number of boundary sites (ancestor sites coupled to it)
 *   sep, bnd   out (may be NULL): site lists in front order, capacities
 *              given by the sizes returned by a first call with NULL
 */
int cl_plan_get_node(const cl_plan* plan, int i, int* parent, int* level, int* n_sep,
                     int* n_bnd, int* sep, int* bnd);

/*
 * cl_plan_check_schedule -- host-side race check of the factorisation's
 * two-stream schedule (panel chain on one stream, bulk updates on the other,
 * ordered only by the events the schedule names).  Replays the factor ops in
 * list order with a vector clock per op and counts, element by element of the
 * fronts and workspace, accesses from different streams that touch one
 * element (at least one writing) without being ordered.  Accesses are the
 * entries that can change a result: GEMM operand rows / columns of unmasked
 * outputs, unmasked copy entries, panel blocks, extend-add map entries.
 *   ignore_waits  1: drop the cross-stream waits (the check then finds races)
 *   conflicts     out: number of unordered conflicting accesses (0 = race-free)
 *   first         out (may be NULL): description of the first one, first_len bytes
 * Works on symbolic plans; needs ~12 bytes of host memory per arena element.
 * Not part of the paper: a verification aid for the schedule.
 */
int cl_plan_check_schedule(const cl_plan* plan, int ignore_waits, long long* conflicts, char* first,
                           int first_len);

/*
 * cl_plan_export -- one of the plan's schedule tables as rows of int64, for
 * host-side checks of the schedule (a test executes the op lists in FP64 on
 * the host and compares with an independent dense inverse).  With out ==
 * NULL only *count (the number of int64 values) is set; otherwise out must
 * hold cap >= *count values.  Row layouts:
 *   CL_TABLE_META        Ns, Nt, V, N, precision, panel, pool_elems,
 *                        tmp_elems, arena_elems, n_levels, perm_ints (the
 *                        permutation workspace per replica, ints)
 *   CL_TABLE_FACTOR_OPS, CL_TABLE_SELINV_OPS
 *                        kind (0 zero, 1 assemble, 2 extend-add, 3 panel,
 *                        4 gemm, 5 copy, 6 gather, 7 extract, 8 row swap of
 *                        the panels [d0, d1), 9 column un-permutation),
 *                        d0, d1, blocks,
 *                        level, stream, wait, signal, digits per operand of a
 *                        digit GEMM (0 otherwise), x0, x1 (a panel op's copy
 *                        descriptors [x0, x1), run by extra CTAs of its
 *                        launch; 0, 0 otherwise)
 *   CL_TABLE_GEMM        a, b, c, lda, ldb, ldc, M, N, K, neg, beta,
 *                        rmask[4], cmask[4], trans (bit 0 A, 1 B, 2 C stored
 *                        transposed)
 *   CL_TABLE_PANEL       a, ld, bp, node, col0, nc (candidate pivot rows: this
 *                        panel's and the next panel's of the supernode),
 *                        lperm, pi (offsets in the permutation workspace of
 *                        the panel's row permutation, which the device
 *                        writes, and of a slot for the supernode's running
 *                        one, which it leaves to host executors), swap_blk0
 *   CL_TABLE_COPY        src, dst, lds, ldd, rows, cols, rmask[4], cmask[4]
 *   CL_TABLE_EXTADD      parent, nfp, nchild, child[2], nfc[2], kc[2], map[2]
 *   CL_TABLE_GATHER      child, parent, nfc, kc, nfp, rs, map
 *   CL_TABLE_MAPS        the site maps of extend-add and gather
 *   CL_TABLE_OFF, CL_TABLE_LD
 *                        offset / leading dimension of the D blocks in the
 *                        fronts, per lattice shape: [V] diagonal, [4V]
 *                        (s, s+nu), [4V] (s+nu, s)
 *   CL_TABLE_SEGMENTS    per lattice shape: Ns, Nt, V, count, pool_base,
 *                        rep_stride, table_base, site_base (replica r of the
 *                        shape has its fronts at pool_base + r rep_stride, its
 *                        tables at table_base, its sites at site_base + r V)
 *   CL_TABLE_VNODES      fronts of the row-vector solves (cl_left_solve), by
 *                        level: front, vec, parent_vec, nf, k, r, level,
 *                        nchild, child_vec[2], child_k[2], ea_map[2], ga_map,
 *                        site0, pan0, npan (vector offsets in complex
 *                        elements per noise vector; parent_vec -1 at a root)
 *   CL_TABLE_VSITES      separator sites of those fronts (front order)
 *   CL_TABLE_UNPERM      per supernode of an un-permutation op: front, nf, k,
 *                        pan0, npan (its panels in CL_TABLE_NODE_PANELS), blk0
 *   CL_TABLE_NODE_PANELS panel indices grouped by supernode, in step order
 * Offsets are elements of one replica's arena; a mask [r0, r1, r2, r3]
 * excludes the indices in [r0, r1) and [r2, r3).  Works on symbolic plans.
 */
enum {
  CL_TABLE_META = 0,
  CL_TABLE_FACTOR_OPS = 1,
  CL_TABLE_SELINV_OPS = 2,
  CL_TABLE_GEMM = 3,
  CL_TABLE_PANEL = 4,
  CL_TABLE_COPY = 5,
  CL_TABLE_EXTADD = 6,
  CL_TABLE_GATHER = 7,
  CL_TABLE_MAPS = 8,
  CL_TABLE_OFF = 9,
  CL_TABLE_LD = 10,
  CL_TABLE_SEGMENTS = 11,
  CL_TABLE_VNODES = 12,
  CL_TABLE_VSITES = 13,
  CL_TABLE_UNPERM = 14,
  CL_TABLE_NODE_PANELS = 15
};
int cl_plan_export(const cl_plan* plan, int table, long long* out, long long cap, long long* count);

/*
 * cl_profile_enable -- enable (1) or disable (0) per-launch timing: while
 * enabled, every compute call records a CUDA event pair on its stream around
 * each kernel launch (this adds event records between launches; use it to
 * attribute time, not for the headline rate).  Enabling clears old records.
 */
int cl_profile_enable(cl_plan* plan, int enable);

/*
 * cl_profile_read -- synchronises on the recorded events and aggregates them
 * per kernel family into out[0..cap-1]; *n receives the number of families.
 */
int cl_profile_read(cl_plan* plan, cl_profile_entry* out, int cap, int* n);

/*
 * cl_profile_trace -- the same records as a timeline: synchronises on them and
 * writes one entry per recorded launch, in issue order, into out[0..cap-1]
 * (*n receives the number of records, which may exceed cap).  Times come from
 * the event pairs on each launch's stream, so the two streams of the
 * factorisation can be compared on one clock; with profiling on, launches do
 * not overlap their predecessors on the same stream (no programmatic launch).
 * CL_ERR_INVALID_ARG for a null plan or n, or a null out with cap > 0.
 */
int cl_profile_trace(cl_plan* plan, cl_trace_entry* out, int cap, int* n);

/*
 * cl_measure_peak -- measures an arithmetic peak of the current device with a
 * throughput kernel (independent FMA / MMA chains on every SM, ~10 ms):
 * unit 0 = FP64 tensor-core MMA (m8n8k4), 1 = FP64 FMA, 2 = FP32 FMA,
 * 3 = BF16 tensor-core MMA (mma.sync m16n8k16, FP32 accumulate),
 * 4 = INT8 tensor-core MMA (mma.sync m16n8k32, INT32 accumulate; "GFLOP/s" = Gop/s).
 * *gflops receives GFLOP/s.  Allocates and frees a small device buffer.
 */
int cl_measure_peak(int unit, double* gflops);

/*
 * Groups: several plans (lattice shapes of uneven size, each with its own
 * batch of replicas) evaluated side by side -- the "ragged" batch of the
 * method's production use -- and the whole fixed schedule captured once into
 * a CUDA graph.
 *
 * cl_group_create -- group of nplans existing plans (not owned: destroy the
 *   group before its plans).  Creates one non-blocking stream per plan.
 * cl_group_drift_eval -- for every plan i: cl_drift_eval(plans[i], links[i],
 *   m, mu, nf, NULL, Gfwd[i], Gbwd[i], Kf[i]) on the plan's own stream, forked
 *   from and joined back into `stream` (arrays of nplans device pointers).
 * cl_group_capture -- captures one cl_group_drift_eval with these pointers
 *   into a CUDA graph (stream capture on an internal stream, so `stream` may
 *   be the legacy default stream; nothing is executed; profiling must be
 *   off).  Later launches read whatever the captured buffers then hold.
 * cl_group_launch -- replays the captured graph on `stream` (one launch).
 */
int cl_group_create(int nplans, cl_plan* const* plans, cl_group** group);
int cl_group_drift_eval(cl_group* group, const double* const* links, double m, double mu, double nf,
                        double* const* Gfwd, double* const* Gbwd, double* const* Kf, cudaStream_t stream);
int cl_group_capture(cl_group* group, const double* const* links, double m, double mu, double nf,
                     double* const* Gfwd, double* const* Gbwd, double* const* Kf, cudaStream_t stream);
int cl_group_launch(cl_group* group, cudaStream_t stream);
void cl_group_destroy(cl_group* group);

/* cl_destroy_plan -- frees the plan and all its device memory (NULL is a no-op). */
void cl_destroy_plan(cl_plan* plan);

/* cl_error_string -- static text for a status code. */
const char* cl_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CLSELINV_H */
