// Internal plan of the selected-inversion library: the nested-dissection
// elimination tree, the front layout in device memory and the fixed launch
// schedule (built once per lattice shape by the host analysis).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "clselinv.h"

namespace cl {

// GEMM tile in complex elements (rows x cols); shared by host schedule and kernels.
constexpr int kTileM = 64;
constexpr int kTileN = 32;
// row swap of the cross-panel pivoting: front columns per CTA (a panel's row
// exchanges are disjoint pairs, swapped in place by several thread groups per
// column)
constexpr int kSwapCols = 64;
// column un-permutation after a supernode's selected-inversion step: front
// rows per CTA (one warp per row)
constexpr int kUnpermRows = 8;
constexpr int kEmuTileM = 128;
// Sites per leaf of the nested dissection and pivoting panel (unknowns) by
// precision.  30 unknowns (10 sites) is the widest panel whose products stay
// single-chunk digit GEMMs (K <= 32 complex); measured on GB300 at 8^3x4 it
// beats 24 and 48 for the emulated-FP64 and FP32 fronts, while the FP64-pipe
// bound native fronts prefer 48.
constexpr int kLeafSites = 8;
constexpr int kPanelFP64 = 48;
constexpr int kPanelFP32 = 30;
constexpr int kPanelEmu = 30;
// digits per operand of the digit GEMMs (CL_FP64_EMU: every product to
// ~2^-58 of its row / column maxima; CL_MIXED_BF16X3: split-BF16x3 Schur and
// off-diagonal selected-inverse products, 7 digits (an FP64 GEMM's accuracy)
// for the panel products with the pivot-block inverse and the diagonal blocks
// of the selected-inverse sweep)
constexpr int kDigitsFP64 = 8;
constexpr int kDigitsMixed = 3;
constexpr int kDigitsDiag = 7;
// precisions whose front GEMMs run on the BF16 tensor cores as digit products
inline bool digit_gemms(int precision) { return precision == CL_FP64_EMU || precision == CL_MIXED_BF16X3; }

// bound of every mbarrier wait of the tensor-core GEMMs (0.5 s); a wait that
// runs out records CL_ERR_TIMEOUT and the kernel drains and leaves
constexpr unsigned long long kDefaultWaitNs = 500000000ull;

struct SNode {
  std::vector<int> sep;       // sites eliminated at this supernode (front order)
  std::vector<int> bnd;       // boundary sites, ordered by position in the parent's front
  std::vector<int> children;
  int parent = -1;
  int level = 0;              // height above the leaves
  int k = 0, r = 0, nf = 0;   // pivot unknowns, boundary unknowns, front order
  int64_t off = 0;            // front offset (elements) in the arena of one replica
  int64_t tmp = 0;            // offset of this front's workspace (elements)
  int ea_map[2] = {-1, -1};   // extend-add site maps of the children (offsets into the plan's maps)
  int ga_map = -1;            // gather site map of this node's boundary (offset into the plan's maps)
};

// One lattice shape of a plan: `count` replicas whose fronts lie in the arena
// at pool_base + r * rep_stride (r < count), with the shape's block tables at
// table_base in the plan's off / ld tables (9 V entries: diagonal, forward,
// backward blocks) and its sites at site_base of the caller's site-indexed
// arrays (links, G blocks, drift: sum of count x V of the earlier shapes).
struct Segment {
  int Ns = 0, Nt = 0, V = 0, count = 0;
  int64_t pool_base = 0, rep_stride = 0, table_base = 0, site_base = 0;
};

// Two excluded index ranges [r0, r1) and [r2, r3) (empty ranges allowed).
struct Mask2 {
  int r0, r1, r2, r3;
  __host__ __device__ bool hit(int i) const { return (i >= r0 && i < r1) || (i >= r2 && i < r3); }
};

// C = beta*C + (neg ? -1 : +1) * A * B on one front; offsets are elements of the
// replica arena; rows in `rmask` and columns in `cmask` of C are left untouched.
struct GemmDesc {
  int64_t a, b, c;
  int lda, ldb, ldc;
  int M, N, K;
  int neg, beta;
  Mask2 rmask, cmask;
  int blk0, tilesN;  // first CTA of this problem inside its launch; tiles along N
  // operands stored transposed (digit-GEMM path only): bit 0 A(i, k) at
  // a + k lda + i, bit 1 B(k, j) at b + j ldb + k, bit 2 C(i, j) at c + j ldc + i
  int trans = 0;
};

// Pivot panel of a supernode: its pivots are chosen among the nc rows col0 ..
// col0 + nc - 1 of the front (the rows of this panel and of the next one in
// the supernode), the chosen rows' block A[pp] (bp x bp, leading dim ld) is
// inverted in place, and the panel's row permutation of those nc rows (lperm:
// position i holds candidate row lperm[i]) is left in the permutation
// workspace, where the row swap applies it to the other columns.  pi: a slot
// of k ints per supernode for its running permutation (position i of the
// front holds the supernode's original row pi[i]), which host executors of
// the exported schedule keep; the device kernels leave it untouched and undo
// the panels' exchanges one by one instead.  swap_blk0: first CTA of the
// panel in the row-swap launch.
struct PanelDesc {
  int64_t a;
  int ld, bp;
  int node, col0;
  int nc;
  int lperm, pi;  // offsets (ints) in the permutation workspace
  int swap_blk0;
};

// After a supernode's step of the selected inversion: the columns of its
// pivot rows are put back in the supernode's original order, G[:, pi[i]] =
// front[:, i] for i < k, on every row of the front, by undoing the panels'
// row exchanges (node_panels[pan0 .. pan0 + npan): its panels in step order)
// in reverse order; one warp per front row.
struct UnpermDesc {
  int64_t front;
  int nf, k;
  int pan0, npan;
  int blk0;
};

// dst[i][j] = src[i][j] for i < rows, j < cols, skipping rows in `rmask` and
// columns in `cmask`.
struct CopyDesc {
  int64_t src, dst;
  int lds, ldd;
  int rows, cols;
  Mask2 rmask, cmask;
  int blk0;
};

// Extend-add (pull form): parent[i][j] += sum_c child_c[kc + 3*map_c[i/3] + i%3][...]
// for both children whose boundary contains the parent sites i/3 and j/3.
struct ExtAddDesc {
  int64_t parent;
  int nfp;
  int nchild;
  int64_t child[2];
  int nfc[2], kc[2];
  int map[2];  // offset into the int map table: parent front site -> child boundary index or -1
  int blk0;
};

// Gather of G_SS (selected inversion): child[kc+i][kc+j] = parent[pos(i)][pos(j)].
struct GatherDesc {
  int64_t child, parent;
  int nfc, kc, nfp, rs;  // rs = boundary sites of the child
  int map;               // offset into the int map table: child boundary index -> parent front site
  int blk0;
};

// Split-digit workspace of one GEMM problem in the FP64-emulation path
// (CL_FP64_EMU): digit tiles of A (7 x Mp x Kp words) and of the real
// embedding of B, transposed (7 x 2 Np x Kp words); chunk exponents
// ([Kp/32][Mp] and [Kp/32][Np] ints); padded sizes.  Output tiles are
// 128 rows x 16 complex columns.
struct EmuDesc {
  int64_t adig, bdig;  // word offsets in the replica's word workspace
  int64_t aexp, bexp;  // int offsets in the replica's int workspace
  int Mp, Np, Kp;      // Mp % 128 == 0, Np % 32 == 0, Kp % 32 == 0 (complex)
  int it0, items;      // split-pass warp items of this problem inside its launch
};


// A front of the row-vector solves w = eta^dag D^{-1} (stochastic estimator):
// per noise vector, the front's vector [J | S] (nf complex) lives at `vec` of
// the forward (R) and backward (W) vector workspaces; the front's factors at
// `front` (A_JJ^{-1} | U-hat on the J rows, -L-hat on the S rows).  Sites of
// the separator (front order) at `site0` of the plan's vsites table (sites
// of the caller's site-indexed arrays; a single-shape plan adds replica x V).
struct VecNode {
  int64_t front, vec, parent_vec;  // parent_vec < 0: root
  int nf, k, r, level;
  int nchild;
  int64_t child_vec[2];
  int child_k[2];
  int ea_map[2], ga_map;
  int site0;
  int blk_nf, blk_r;  // first CTA of this node in a level launch over nf / r elements (tiles of 128)
  int pan0, npan;     // the supernode's panels (node_panels), whose row exchanges the solve undoes
};

enum OpKind { OP_ZERO, OP_ASSEMBLE, OP_EXTADD, OP_PANEL, OP_GEMM, OP_COPY, OP_GATHER, OP_EXTRACT, OP_SWAP, OP_UNPERM };

// One scheduled launch.  The factorisation runs on two streams: the
// critical chain (panel inverses, panel products, next-panel strips) on the
// caller's stream (stream 0) and the bulk rank-b updates with the panel
// write-back on an internal stream (stream 1).  `wait` names an earlier op on
// the other stream whose completion must precede this one (-1: none);
// `signal` records the completion event of this op.
struct Op {
  OpKind kind;
  int d0, d1;     // descriptor range in the table of this kind
  int blocks;     // CTAs per replica
  int level;
  int stream = 0;
  int wait = -1;
  bool signal = false;
  bool single_chunk = false;  // digit GEMM with every K <= 32: persistent kernel
  int ndig = 0;               // digit GEMM: base-256 digits per operand (3, 7 or 8)
  // panel op: copy descriptors [x0, x1) (xblocks blocks of 256 entries) run by
  // extra CTAs of the panel launch, beside the panel inverses
  int x0 = 0, x1 = 0, xblocks = 0;
  bool pdl = false;           // set at launch: the op's first kernel follows a kernel of its stream directly
};

struct Plan {
  // a single-shape plan: Ns, Nt, V of the lattice, batch replicas (grid.y of
  // every front launch, one arena_elems block per replica); a ragged plan
  // (several shapes, cl_analyze_ragged): V = sites of all lattices, batch =
  // number of lattices, fbatch = 1, every front of every lattice at its own
  // offset in one arena and in the same launches
  int Ns = 0, Nt = 0, V = 0, N = 0, batch = 0, precision = CL_FP64;
  int fbatch = 1;             // grid.y of the front launches (replicas sharing the descriptors)
  bool ragged = false;
  std::vector<Segment> segs;  // lattice shapes: the per-site kernels run once per segment
  int panel = kPanelFP64;
  bool has_device = false;
  int device = 0;
  int num_sms = 0;            // multiprocessors of the device (set up with the device state)
  int chain_sms = 2;          // SMs the bulk digit GEMMs leave to the panel chain (two-stream plans)
  unsigned long long wait_ns = kDefaultWaitNs;  // limit of the GEMM roles' mbarrier waits (cl_plan_set_wait_limit)
  std::vector<SNode> nodes;   // postorder, root last
  int n_levels = 0;
  double factor_flops = 0, selinv_flops = 0;
  int64_t pool_elems = 0;     // fronts, per replica
  int64_t tmp_elems = 0;      // workspace, per replica
  int64_t arena_elems = 0;    // per replica (pool + workspace, padded)
  // host tables
  std::vector<int64_t> off_diag, off_fwd, off_bwd;  // assembly / extraction offsets (single shape)
  std::vector<int> ld_diag, ld_fwd, ld_bwd;
  std::vector<int64_t> off_all;                     // per segment: diagonal | forward | backward
  std::vector<int> ld_all;
  std::vector<int> maps;                            // int maps of extend-add and gather
  std::vector<GemmDesc> gemm;
  std::vector<PanelDesc> panels;
  std::vector<UnpermDesc> unperm;
  std::vector<int> node_panels;  // panel indices grouped by supernode, in step order
  int64_t perm_ints = 0;         // permutation workspace per replica (ints)
  std::vector<CopyDesc> copies;
  std::vector<ExtAddDesc> extadd;
  std::vector<GatherDesc> gather;
  std::vector<EmuDesc> emu;                         // parallel to gemm (CL_FP64_EMU only)
  int64_t emu_words = 0, emu_ints = 0;              // workspace per replica
  std::vector<Op> factor_ops, selinv_ops;
  // row-vector solves of the stochastic estimator: nodes sorted by level,
  // vlevel[h] .. vlevel[h+1] the nodes of level h; CTAs per level launch
  std::vector<VecNode> vnodes;
  std::vector<int> vsites, vlevel, vblk_nf, vblk_r;
  int64_t vec_elems = 0;  // complex elements of one front-vector workspace per noise vector and replica
  // device memory
  void* d_arena = nullptr;       // batch * arena_elems complex (precision-dependent)
  int* d_status = nullptr;       // [4]: code, node, column, pivot growth (float bits)
  int64_t* d_off = nullptr;      // off_diag | off_fwd | off_bwd
  int* d_ld = nullptr;           // ld_diag | ld_fwd | ld_bwd
  int* d_maps = nullptr;
  GemmDesc* d_gemm = nullptr;
  PanelDesc* d_panels = nullptr;
  UnpermDesc* d_unperm = nullptr;
  int* d_node_panels = nullptr;
  int* d_perm = nullptr;  // fbatch x perm_ints
  CopyDesc* d_copies = nullptr;
  ExtAddDesc* d_extadd = nullptr;
  GatherDesc* d_gather = nullptr;
  EmuDesc* d_emu = nullptr;
  VecNode* d_vnodes = nullptr;
  int* d_vsites = nullptr;
  unsigned* d_emu_words = nullptr;
  int* d_emu_ints = nullptr;
  // Langevin-step buffers (all replicas): G blocks, drift, link inverses,
  // cooling fields, reduction partials and max slots
  double* d_Gdiag = nullptr;
  double* d_Gfwd = nullptr;
  double* d_Gbwd = nullptr;
  double* d_K = nullptr;
  double* d_Ui = nullptr;
  double* d_F = nullptr;
  double* d_Om = nullptr;
  double* d_Omi = nullptr;
  double* d_part = nullptr;
  unsigned long long* d_slots = nullptr;
  size_t device_bytes = 0;
  int launches_per_eval = 0;
  // per-launch timing (cl_profile_enable)
  struct ProfRec {
    int family;
    void* ev0;
    void* ev1;
    double flops, bytes;
    int phase = -1, op = -1, stream = 0, level = -1;  // op list (0 factor, 1 selected inversion), index, stream
  };
  bool profiling = false;
  std::vector<ProfRec> prof;
  // the factorisation's two streams (0: high-priority panel chain, 1: bulk
  // updates) and the events of its cross-stream dependencies, created with
  // the device state
  void* streams[2] = {nullptr, nullptr};
  std::vector<void*> op_events;  // per factor op (nullptr when it does not signal)
  void* fork_event = nullptr;
  void* join_events[2] = {nullptr, nullptr};
  int prio_lo = 0, prio_hi = 0;  // the device's lowest / highest stream priority
};

// kernel families for profiling records
enum Family { F_ZERO, F_ASSEMBLE, F_EXTADD, F_PANEL, F_GEMM, F_COPY, F_GATHER, F_EXTRACT, F_DRIFT, F_COUNT };

// host analysis (analyze.cpp); throws std::invalid_argument on invalid input.
// panel: pivoting panel width in unknowns (multiple of 3, 3..48), 0 = default
void analyze_host(Plan& p, int Ns, int Nt, int batch, int precision, int panel = 0);
// several shapes (count[i] lattices of Ns[i]^3 x Nt[i]) in one merged schedule
void analyze_ragged(Plan& p, int nshapes, const int* Ns, const int* Nt, const int* count, int precision,
                    int panel = 0);
// number of unordered conflicting element accesses between the two streams of
// the factor schedule (0: race-free); ignore_waits drops the cross-stream
// waits (the check must then find races); *first describes the first one
long long check_factor_schedule(const Plan& p, bool ignore_waits, std::string* first);

}  // namespace cl
