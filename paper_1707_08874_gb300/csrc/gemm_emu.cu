// FP64-accurate complex GEMM on the BF16 tensor cores (precision CL_FP64_EMU).
//
// GB300's FP64 pipe delivers ~1.1 TFLOP/s; its BF16 tensor cores, driven by
// tcgen05, two orders of magnitude more.  Each FP64 operand is written exactly
// as
//   a = sign * 2^e * sum_{p=1..7} d_p 2^{-8p} + (truncation < 2^{e-56}),
// with integer digits 0 <= d_p <= 255 (exact in BF16) and one exponent e per
// row (A) or column (B) and per chunk of 32 complex k.  The product is the sum
// over digit pairs p + q <= 6 (0-based: 28 BF16 products, 7 levels p + q) of
// integer dot products: exact in the FP32 accumulator for the leading levels
// (sums < 2^24) and rounded below FP64 resolution for the others.  Level sums
// are scaled by powers of two and accumulated across chunks in triple-float
// (three FP32 words, error-free two-sums), relative to the largest row /
// column exponent; FP64 arithmetic appears only in the epilogue (two
// additions per output).  Accuracy equals an FP64 GEMM to within a small
// factor (numpy emulation of the same digits and roundings: normwise relative
// error 4e-16 - 1.1e-15 against 5e-16 - 1e-15 for FP64).
//
// Complex products are one real product of twice the size: A is the real
// M x 2K matrix of interleaved (re, im) pairs, B is expanded into the real
// 2K x 2N matrix of [[br, bi], [-bi, br]] blocks by the split pass.
//
// Two kernels per GEMM launch:
//   k_emu_split    digits and exponents of A and B, written as tiles in the
//                  order the tensor core reads shared memory;
//   k_gemm_emu_persist / k_gemm_emu_chunked  the digit products as tcgen05
//                  MMAs with FP32 accumulators in tensor memory, the fold and
//                  the FP64 epilogue (single-chunk and chunked launches).
#include <algorithm>
#include <cstring>

#include "kernels.cuh"

namespace cl {
namespace {

// base-256 digits per operand (ND, a template parameter of the kernels):
// 8 for the FP64 fronts (products accurate to ~2^-58 of the row / column
// maxima, well below FP64 rounding of the result), 7 for the stand-alone
// GEMM (an FP64 GEMM's accuracy), 3 for the split-BF16x3 Schur products
// (FP32-class accuracy)
constexpr int kChunk = 32;   // complex k per exponent chunk (64 real k)
constexpr int kTileCx = 16;  // complex columns of C per CTA (32 real columns of B')

__device__ __forceinline__ int exp_of(double v) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? -2000 : E - 1023;  // zero / subnormal count as absent
}

// BF16 bit patterns of the ND digits of |v| 2^{-e} (< 1), truncated to a
// window of 8 ND bits, with v's sign
template <int ND>
__device__ __forceinline__ void digits(double v, int e, unsigned short (&d)[ND]) {
  static_assert(ND >= 2 && ND <= 8, "8 ND bits must fit the 64-bit window");
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned short sgn = b < 0 ? 0x8000u : 0u;
  unsigned long long X = 0;
  if (E != 0 && E != 0x7FF) {
    const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (E - 1023) + (8 * ND - 52) - e;  // X = m 2^sh = |v| 2^{8 ND - e} < 2^{8 ND}
    if (sh >= 0) X = m << sh;
    else if (sh > -64) X = m >> (-sh);
  }
#pragma unroll
  for (int p = 0; p < ND; ++p) {
    const unsigned dg = (unsigned)(X >> (8 * (ND - 1 - p))) & 0xFFu;
    d[p] = dg ? (unsigned short)((__float_as_uint((float)dg) >> 16) | sgn) : (unsigned short)0;
  }
}

// Digit tiles, laid out for the tensor core's no-swizzle K-major operand
// format: 16-k slabs; inside a slab, 8-row groups of two 8 x 8 core matrices
// (k 0-7, 8-15), each core matrix 8 rows of 16 bytes (256 bytes per group).
// With ND digits per operand:
//   A: per (128-row block, chunk) one 16 ND KB block [digit p][slab][16 groups]
//      (4096 words per digit).
//   B': per (32-real-column block, chunk) one 4 ND KB block [slab][digit q][4
//      groups] (256 ND words per slab): in a slab the digits' rows follow one
//      another at the uniform 256-byte group stride, so one MMA of width
//      N = 32 (ND - p) multiplies A digit p by B' digits q = 0 .. ND-1-p at once.
// Word (two BF16: re / im of one complex k) of A row `row`, lane = complex k
// in the chunk:
template <int ND>
__device__ __forceinline__ int64_t a_tile_word(const EmuDesc& e, int nch, int p, int row, int c, int lane) {
  const int64_t blk = (int64_t)(row / 128) * nch + c;
  const int r = row & 127;
  return e.adig + (blk * ND + p) * 4096 + (lane >> 3) * 1024 + (r >> 3) * 64 + ((lane >> 2) & 1) * 32 + (r & 7) * 4 +
         (lane & 3);
}
// ... and of B' row (real column of the embedding) `nreal`:
template <int ND>
__device__ __forceinline__ int64_t b_tile_word(const EmuDesc& e, int nch, int q, int nreal, int c, int lane) {
  const int64_t blk = (int64_t)(nreal / 32) * nch + c;
  const int r = nreal & 31;
  return e.bdig + blk * (1024 * ND) + (lane >> 3) * (256 * ND) + q * 256 + (r >> 3) * 64 + ((lane >> 2) & 1) * 32 +
         (r & 7) * 4 + (lane & 3);
}

// Split pass: one warp per item.  A items (row, chunk): lanes take the 32
// complex k of the chunk and write (re, im) digit pairs.  B items (complex
// column n, chunk): lanes take the chunk's 32 k; the real embedding of
// b = br + i bi is written directly as two rows of B'^T:
//   row 2n   : (br, -bi)   (real column 2n of [[br, bi], [-bi, br]] per k)
//   row 2n+1 : (bi,  br)
// Padding (rows >= M, columns >= N, k >= K) gets zero digits.
template <int ND>
__global__ void __launch_bounds__(256) k_emu_split(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed,
                                                   int d0, int d1, const double2* __restrict__ arena,
                                                   int64_t stride, unsigned* __restrict__ words,
                                                   int* __restrict__ ints, int64_t wstride, int64_t istride,
                                                   int total, int* __restrict__ status) {
  pdl_enter();
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= total) return;
  int lo = d0, hi = d1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ed[mid].it0 <= item) lo = mid;
    else hi = mid - 1;
  }
  const GemmDesc g = gd[lo];
  const EmuDesc e = ed[lo];
  const double2* base = arena + blockIdx.y * stride;
  unsigned* W = words + blockIdx.y * wstride;
  int* I = ints + blockIdx.y * istride;
  const int nch = e.Kp / kChunk;
  int it = item - e.it0;
  const int nA = e.Mp * nch;
  const bool isA = it < nA;
  if (!isA) it -= nA;
  const int line = it / nch, c = it % nch;  // row (A) or complex column (B)
  const int k = c * kChunk + lane;
  double2 v = make_double2(0, 0);
  if (isA) {
    if (line < g.M && k < g.K)
      v = base[g.a + ((g.trans & 1) ? (int64_t)k * g.lda + line : (int64_t)line * g.lda + k)];
  } else {
    if (line < g.N && k < g.K)
      v = base[g.b + ((g.trans & 2) ? (int64_t)line * g.ldb + k : (int64_t)k * g.ldb + line)];
  }
  // an infinite or NaN operand has no digits: report it instead of dropping it
  if (!isfinite(v.x) || !isfinite(v.y)) set_status(status, CL_ERR_NONFINITE, -1, -1);
  int ex = max(exp_of(v.x), exp_of(v.y));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
  const int ee = ex + 1;
  unsigned short dr[ND], di[ND];
  digits<ND>(v.x, ee, dr);
  digits<ND>(v.y, ee, di);
  if (isA) {
    if (lane == 0) I[e.aexp + (int64_t)c * e.Mp + line] = ee;
#pragma unroll
    for (int p = 0; p < ND; ++p)
      W[a_tile_word<ND>(e, nch, p, line, c, lane)] = (unsigned)dr[p] | ((unsigned)di[p] << 16);
  } else {
    if (lane == 0) I[e.bexp + (int64_t)c * e.Np + line] = ee;
#pragma unroll
    for (int p = 0; p < ND; ++p) {
      W[b_tile_word<ND>(e, nch, p, 2 * line, c, lane)] =
          (unsigned)dr[p] | ((unsigned)(di[p] ^ (di[p] ? 0x8000u : 0u)) << 16);
      W[b_tile_word<ND>(e, nch, p, 2 * line + 1, c, lane)] = (unsigned)di[p] | ((unsigned)dr[p] << 16);
    }
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float pow2f(int k) { return k < -126 ? 0.f : __int_as_float((k + 127) << 23); }

// f * 2^ex as a double, built from the float's bits with integer operations
// (exact; the FP64 pipe is GB300's scarcest unit).  Zero / subnormal floats
// and results below the double range give 0; sign flipped when neg.
__device__ __forceinline__ double f2d_scaled(float f, int ex, bool neg) {
  const unsigned u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 0xFFu);
  if (e == 0) return 0.0;
  const int ed = e - 127 + 1023 + ex;
  if (ed <= 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)((u >> 31) ^ (neg ? 1u : 0u)) << 63;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)ed << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// Two adjacent complex values (32 bytes, 32-byte aligned) in one 256-bit
// global access: a whole sector per lane
__device__ __forceinline__ void ld_c2(const double2* p, double2& a, double2& b) {
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a.x), "=d"(a.y), "=d"(b.x), "=d"(b.y) : "l"(p));
}
__device__ __forceinline__ void st_c2(double2* p, double2 a, double2 b) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a.x), "d"(a.y), "d"(b.x), "d"(b.y)
               : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05 building blocks of the digit GEMMs.  Operands reach shared memory by
// bulk copies of the pre-tiled digit planes; one thread issues BF16 MMAs into
// FP32 accumulators in tensor memory (one 32-column accumulator per level
// p + q, 224 columns per set); warps read the levels back with tcgen05.ld.
// Every wait on an mbarrier gives up after a bounded time, records
// CL_ERR_TIMEOUT, waits once more for what it had in flight and leaves through
// the normal teardown (tensor memory freed).
constexpr int kAHalf = 8192;     // bytes: 128 rows x 32 real k, BF16 (two 16-k slabs)
constexpr int kBHalf = 2048;     // bytes per digit: 32 real columns x 32 real k
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28;
// M = 128, N = 32 (ND - p) for A digit p (a multiple of 16, <= 256)
constexpr uint32_t kTcIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);
__host__ __device__ constexpr uint32_t tc_idesc(int nd, int p) {
  return kTcIdescBase | ((uint32_t)(4 * (nd - p)) << 17);
}
// bound of the waits that drain copies and MMAs in flight before a CTA
// leaves (always the full bound; the role waits take the launch's limit,
// kDefaultWaitNs unless a test shortens it)
constexpr unsigned long long kWaitNs = kDefaultWaitNs;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// bounded wait for the completion of phase `parity`; false after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
  const unsigned long long t0 = gtimer();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, unsigned bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory matrix descriptor, no swizzle, K-major: core matrices 8 rows
// x 16 bytes; 128 bytes between the two core matrices of a 16-k slab (k
// direction), 256 bytes between 8-row groups; descriptor version 1 (bit 46)
__device__ __forceinline__ unsigned long long umma_desc(uint32_t saddr) {
  return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(256 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, unsigned long long ad, unsigned long long bd, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// load without waiting: several loads, then one tmem_ld_wait()
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&v)[16]) { tmem_ld16_issue(taddr, v); }
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&v)[8]) { tmem_ld8_issue(taddr, v); }
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Persistent digit GEMM for launches whose problems all have K <= 32 (one
// exponent chunk: the sweep updates of the factorisation and the panel
// products).  One CTA per SM takes a contiguous range of output tiles (128
// rows x 16 complex columns) of the launch; warp-specialised, 64 + 128 NG threads:
//   warp 0 lane 0  producer: bulk copies of the current row block's A digits
//                  (112 KB, kept while consecutive tiles share the block) and
//                  of each tile's B' digits into a two-stage ring (28 KB);
//   warp 1 lane 0  MMA issuer: per tile 28 tcgen05 MMAs (per A digit p and
//                  16-k slab, one 128 x 32(7-p) x 16 product with B' digits
//                  0 .. 6-p) into one of two accumulator sets in tensor memory
//                  (7 levels x 32 columns at TMEM columns 0 and 256), so the
//                  MMAs of tile i+1 run while tile i is folded and written;
//   warps 2-17     fold (thread = row) and FP64 epilogue in NG = 4 groups of
//                  four warps (2 with CLSELINV_FOLD_GROUPS=2), each owning
//                  16/NG of every tile's complex columns: four warps per
//                  scheduler hide the latency of the fold's dependent FP32
//                  chains and of the write-back's FP64 additions, and a
//                  tile's fold and write-back take 1/NG as long as with one
//                  group per tile (the panel chain's small launches have one
//                  tile per CTA); the C row segment is prefetched into L1.
// With one chunk the row / column exponents are the chunk's own, the fold
// scale is 2^{-16-8L} and the output exponent e_row + f_col.
constexpr int kPA = 16384;  // bytes: one A digit tile, 128 rows x 64 real k
constexpr int kPB = 4096;   // bytes: one B' digit tile, 32 real columns x 64 real k
constexpr int kPCtl = 1024;
__host__ __device__ constexpr size_t p_smem_bytes(int nd) { return (size_t)nd * kPA + 2 * (size_t)nd * kPB + kPCtl; }
constexpr uint32_t kPCols = 512;

// tile t of the launch -> problem, row block and 16-column tile
struct TileRef {
  int di, rb, j;
};
__device__ __forceinline__ TileRef tile_ref(const GemmDesc* __restrict__ gd, int d0, int d1, int t) {
  TileRef r;
  r.di = find_desc(gd, d0, d1, t);
  const int rel = t - gd[r.di].blk0, tn = gd[r.di].tilesN;
  r.rb = rel / tn;
  r.j = rel - r.rb * tn;
  return r;
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, unsigned parity, const volatile int* abort_flag,
                                             unsigned long long limit_ns) {
  const unsigned long long t0 = gtimer();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort_flag || gtimer() - t0 > limit_ns) return false;
  }
}

template <int NG, int ND>  // fold groups of four warps, digits per operand
__global__ void __launch_bounds__(64 + 128 * NG, 1)
    k_gemm_emu_persist(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed, int d0, int d1, int total,
                       double2* __restrict__ arena, int64_t stride, const unsigned* __restrict__ words,
                       const int* __restrict__ ints, int64_t wstride, int64_t istride, int* __restrict__ status,
                       unsigned long long wait_ns) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem_p[];
  unsigned char* sA = smem_p;                   // [7][kPA]
  unsigned char* sB = smem_p + ND * kPA;        // [2 stages][ND][kPB]
  unsigned char* ctl = sB + 2 * ND * kPB;
  // mbarriers: [0] A landed, [1,2] B stage landed, [3,4] B stage consumed,
  //            [5,6] accumulator set full, [7,8] accumulator set drained
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ctl);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 96);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 100);
  const uint32_t bar0 = smem_u32(bars);
  auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
  const uint32_t b_afull = bar0;

  const int G = gridDim.x;
  const int t0 = (int)((int64_t)total * blockIdx.x / G), t1 = (int)((int64_t)total * (blockIdx.x + 1) / G);
  const int n = t1 - t0;
  const unsigned* Wd = words + blockIdx.y * wstride;
  const int* Id = ints + blockIdx.y * istride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kPCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < 7; ++i) mbar_init(bar(i), 1);
    mbar_init(bar(7), 128 * NG);  // every fold group drains an accumulator set
    mbar_init(bar(8), 128 * NG);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      int prev = -1, issued = 0, a_loads = 0;
      bool good = true;
      for (int i = 0; i < n && good && !*abort_flag; ++i) {
        const TileRef tr = tile_ref(gd, d0, d1, t0 + i);
        const EmuDesc& e = ed[tr.di];
        const int key = tr.di * 65536 + tr.rb;
        if (key != prev) {
          // the MMAs of the previous tile read the old A block: wait for them
          if (i > 0 && !mbar_wait_ab(bar(3 + ((i - 1) & 1)), ((i - 1) >> 1) & 1, abort_flag, wait_ns)) {
            good = false;
            break;
          }
          mbar_expect_tx(b_afull, (unsigned)(ND * kPA));
          for (int p = 0; p < ND; ++p)
            bulk_g2s(smem_u32(sA + p * kPA), Wd + e.adig + ((int64_t)tr.rb * ND + p) * 4096, kPA, b_afull);
          ++a_loads;
          prev = key;
        }
        const int s = i & 1, u = i >> 1;
        if (i >= 2 && !mbar_wait_ab(bar(3 + s), (u - 1) & 1, abort_flag, wait_ns)) {
          good = false;
          break;
        }
        mbar_expect_tx(bar(1 + s), (unsigned)(ND * kPB));
        bulk_g2s(smem_u32(sB + s * ND * kPB), Wd + e.bdig + (int64_t)tr.j * (1024 * ND), ND * kPB, bar(1 + s));
        issued = i + 1;
      }
      if (!good) {
        *abort_flag = 1;
        set_status(status, CL_ERR_TIMEOUT, -5, t0);
      }
      if (*abort_flag) {  // copies still in flight: the last two stages and the A block, bounded
        for (int i = max(0, issued - 2); i < issued; ++i) mbar_wait(bar(1 + (i & 1)), (i >> 1) & 1);
        if (a_loads > 0) mbar_wait(b_afull, (a_loads - 1) & 1);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      int prev = -1, a_use = 0, last = -1;
      bool good = true;
      const uint32_t a0 = smem_u32(sA);
      for (int i = 0; i < n && good && !*abort_flag; ++i) {
        const TileRef tr = tile_ref(gd, d0, d1, t0 + i);
        const int key = tr.di * 65536 + tr.rb;
        if (key != prev) {
          if (!mbar_wait_ab(b_afull, a_use & 1, abort_flag, wait_ns)) {
            good = false;
            break;
          }
          ++a_use;
          prev = key;
        }
        const int s = i & 1, u = i >> 1;
        if (!mbar_wait_ab(bar(1 + s), u & 1, abort_flag, wait_ns) ||
            (i >= 2 && !mbar_wait_ab(bar(7 + s), (u - 1) & 1, abort_flag, wait_ns))) {
          good = false;
          break;
        }
        tc_fence_after();
        const uint32_t b0 = smem_u32(sB + s * ND * kPB), d = tmem + 256u * s;
#pragma unroll 1
        for (int p = 0; p < ND; ++p)
#pragma unroll
          for (int kb = 0; kb < 4; ++kb)
            umma_bf16(d + 32 * p, umma_desc(a0 + p * kPA + kb * 4096), umma_desc(b0 + kb * (ND * 1024)),
                      tc_idesc(ND, p), (p | kb) != 0 ? 1u : 0u);
        umma_commit(bar(3 + s));
        umma_commit(bar(5 + s));
        last = i;
      }
      if (!good) {
        *abort_flag = 1;
        set_status(status, CL_ERR_TIMEOUT, -6, t0);
      }
      if (*abort_flag && last >= 0) mbar_wait(bar(5 + (last & 1)), (last >> 1) & 1);  // MMAs in flight
    }
    __syncwarp();
  } else {  // ---- fold and epilogue: thread = row; group g (warps 2+4g .. 5+4g) owns complex columns CC g .. CC g + CC-1
    constexpr int CR = 32 / NG, CC = CR / 2;  // real / complex columns of a group
    const int grp = (warp - 2) >> 2, q4 = warp & 3, rl = q4 * 32 + lane;
    int prev = -1, erow = 0;
    for (int i = 0; i < n; ++i) {
      __syncwarp();
      if (__any_sync(0xffffffffu, *abort_flag)) break;
      const TileRef tr = tile_ref(gd, d0, d1, t0 + i);
      const GemmDesc g = gd[tr.di];
      const int64_t bexp = ed[tr.di].bexp;
      const int key = tr.di * 65536 + tr.rb;
      if (key != prev) {
        erow = Id[ed[tr.di].aexp + tr.rb * 128 + rl];
        prev = key;
      }
      const int r = tr.rb * 128 + rl, col0 = tr.j * kTileCx;
      const bool row_ok = r < g.M && !g.rmask.hit(r);
      const bool neg = g.neg != 0;
      const bool ctr = (g.trans & 4) != 0;  // C stored transposed: column stride ldc
      const int64_t cs = ctr ? g.ldc : 1;
      double2* crow = arena + blockIdx.y * stride + g.c + (ctr ? (int64_t)r : (int64_t)r * g.ldc) + col0 * cs;
      // this group's column exponents and C row segment, loaded while the MMAs run
      const int c8 = col0 + CC * grp;
      int fe[CC];
      {
        const int4* fp = reinterpret_cast<const int4*>(Id + bexp + c8);
#pragma unroll
        for (int q = 0; q < CC / 4; ++q) {
          const int4 x = fp[q];
          fe[4 * q] = x.x, fe[4 * q + 1] = x.y, fe[4 * q + 2] = x.z, fe[4 * q + 3] = x.w;
        }
      }
      // this group's C row segment; untransposed and 32-byte aligned (every
      // lane of a warp, when ldc is even), it moves two columns per access
      double2* cseg = crow + CC * grp * cs;
      const bool wide = !ctr && (reinterpret_cast<uintptr_t>(cseg) & 31u) == 0;
      double2 cv[CC];
      if (row_ok && g.beta) {
#pragma unroll
        for (int jj = 0; jj < CC; jj += 2) {
          if (wide && c8 + jj + 1 < g.N) {
            ld_c2(cseg + jj, cv[jj], cv[jj + 1]);
          } else {
            cv[jj] = c8 + jj < g.N ? cseg[jj * cs] : make_double2(0, 0);
            cv[jj + 1] = c8 + jj + 1 < g.N ? cseg[(jj + 1) * cs] : make_double2(0, 0);
          }
        }
      }
      const int s = i & 1, u = i >> 1;
      const bool got = mbar_wait_ab(bar(5 + s), u & 1, abort_flag, wait_ns);
      if (!__all_sync(0xffffffffu, got)) {
        if (!*abort_flag) set_status(status, CL_ERR_TIMEOUT, -7, t0);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      {  // this group's CC complex columns (CR TMEM columns per level)
        const int hh = grp;
        float h[CR], mi[CR], lo[CR];
        const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + 256u * s + CR * hh;
        {  // levels 0-3: four loads, one wait
          constexpr int N1 = ND < 4 ? ND : 4;
          uint32_t v[N1][CR];
#pragma unroll
          for (int L = 0; L < N1; ++L) tmem_ld_issue(ta + 32 * L, v[L]);
          tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < CR; ++k) {
            h[k] = __uint_as_float(v[0][k]) * 0x1p-16f;
            two_sum(h[k], __uint_as_float(v[1][k]) * 0x1p-24f, h[k], mi[k]);
            lo[k] = 0.f;
#pragma unroll
            for (int L = 2; L < N1; ++L) {
              float s2, e2;
              two_sum(mi[k], __uint_as_float(v[L][k]) * __int_as_float((127 - 16 - 8 * L) << 23), s2, e2);
              mi[k] = s2;
              lo[k] += e2;
            }
          }
        }
        if constexpr (ND > 4) {  // levels 4 .. ND-1, at most 2^-32 of the leading level
          // with 8 digits level 4 enters by one error-free addition of its own;
          // the remaining levels (>= 2^-40 below the leading level with 8
          // digits, >= 2^-32 with 7) are summed in FP32 and enter by one more
          constexpr int N2 = ND - 4, E2 = ND >= 8 ? 1 : 0;
          uint32_t v[N2][CR];
#pragma unroll
          for (int L = 0; L < N2; ++L) tmem_ld_issue(ta + 32 * (L + 4), v[L]);
          tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < CR; ++k) {
            float s2, e2;
            if (E2) {
              two_sum(mi[k], __uint_as_float(v[0][k]) * 0x1p-48f, s2, e2);
              mi[k] = s2;
              lo[k] += e2;
            }
            float x = __uint_as_float(v[E2][k]) * __int_as_float((127 - 48 - 8 * E2) << 23);
#pragma unroll
            for (int L = E2 + 1; L < N2; ++L)
              x = fmaf(__uint_as_float(v[L][k]), __int_as_float((127 - 48 - 8 * L) << 23), x);
            two_sum(mi[k], x, s2, e2);
            mi[k] = s2;
            lo[k] += e2;
          }
        }
        tc_fence_before();
        mbar_arrive(bar(7 + s));  // this group is done with accumulator set s
        if (!row_ok) continue;
#pragma unroll
        for (int jj = 0; jj < CC; jj += 2) {
          double2 vp[2];
          bool okc[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int j2 = jj + q, cc = c8 + j2;
            okc[q] = cc < g.N && !g.cmask.hit(cc);
            const int ex = erow + fe[j2];
            double vv[2];
#pragma unroll
            for (int part = 0; part < 2; ++part) {
              const int k = 2 * j2 + part;
              float s1, e1;
              two_sum(h[k], mi[k], s1, e1);
              vv[part] = f2d_scaled(s1, ex, neg) + f2d_scaled(e1 + lo[k], ex, neg);
            }
            vp[q] = make_double2(vv[0], vv[1]);
            if (g.beta) vp[q] = cadd(vp[q], cv[j2]);
          }
          if (wide && okc[0] && okc[1]) {
            st_c2(cseg + jj, vp[0], vp[1]);
          } else {
            if (okc[0]) cseg[jj * cs] = vp[0];
            if (okc[1]) cseg[(jj + 1) * cs] = vp[1];
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Persistent digit GEMM for chunked launches (some K > 32: the products of the
// selected inversion, K up to a pivot block).  One CTA per SM over the output
// tiles (128 rows x 16 complex columns) t = blockIdx.x, + gridDim.x, ...; per
// tile its chunks of 32 complex k in order, each chunk in two halves of 32
// real k.  Warp-specialised, 64 + 128 NG threads:
//   warp 0 lane 0  producer: per half, the ND A digit half-tiles (8 KB each)
//                  and the B' half-block (2 ND KB) into a ring of three
//                  stages (two with 8 digits);
//   warp 1 lane 0  MMA issuer: 2 ND wide MMAs per half into one of two TMEM
//                  accumulator sets (set = chunk parity), so the MMAs of
//                  chunk k+1 run while chunk k is folded;
//   warps 2-9      fold: NG = 2 groups of four warps, group g owning complex
//                  columns 8g .. 8g+7 of the tile (thread = row), fold each
//                  chunk's levels into triple-float with the chunk's row /
//                  column exponents and write the tile after its last chunk
//                  (four groups, 96 registers with spills, measured ~1%
//                  slower on the selected inversion).
// ring stage of ND digits (bytes) and stages (8 digits: two, to stay within
// the 227 KB of shared memory of a CTA)
__host__ __device__ constexpr int c_stage_bytes(int nd) { return nd * (kAHalf + kBHalf); }
__host__ __device__ constexpr int c_stages(int nd) { return nd >= 8 ? 2 : 3; }
__host__ __device__ constexpr size_t c_smem_bytes(int nd) { return (size_t)c_stages(nd) * c_stage_bytes(nd) + 1024; }
constexpr int kChunkedGroups = 2;  // fold groups of the chunked kernel

template <int NG, int ND>  // fold groups of four warps, digits per operand
__global__ void __launch_bounds__(64 + 128 * NG, 1)
    k_gemm_emu_chunked(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed, int d0, int d1, int total,
                       double2* __restrict__ arena, int64_t stride, const unsigned* __restrict__ words,
                       const int* __restrict__ ints, int64_t wstride, int64_t istride, int* __restrict__ status,
                       unsigned long long wait_ns) {
  pdl_enter();
  constexpr int kCStage = c_stage_bytes(ND), kCStages = c_stages(ND);
  extern __shared__ __align__(1024) unsigned char smem_c[];
  unsigned char* ctl = smem_c + kCStages * kCStage;
  // mbarriers: [0..2] stage landed, [3..5] stage consumed (the first
  //            kCStages of each), [6,7] accumulator set full, [8,9]
  //            accumulator set drained
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ctl);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 96);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 100);
  const uint32_t bar0 = smem_u32(bars);
  auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
  auto stageA = [&](int s) { return smem_c + s * kCStage; };
  auto stageB = [&](int s) { return smem_c + s * kCStage + ND * kAHalf; };

  // tiles are dealt round-robin (tile t to CTA t mod G): the CTAs then work
  // on neighbouring tiles at any moment, so the row blocks of A and column
  // blocks of B' in flight stay few and are served from L2 (each tile streams
  // every chunk of its operands; a contiguous range per CTA would stream all
  // row blocks at once)
  const int G = gridDim.x;
  const int t0 = blockIdx.x, t1 = total;
  const unsigned* Wd = words + blockIdx.y * wstride;
  const int* Id = ints + blockIdx.y * istride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kPCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < 8; ++i) mbar_init(bar(i), 1);
    mbar_init(bar(8), 128 * NG);  // every fold group drains a set
    mbar_init(bar(9), 128 * NG);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      int q = 0;
      bool good = true;
      for (int t = t0; t < t1 && good && !*abort_flag; t += G) {
        const TileRef tr = tile_ref(gd, d0, d1, t);
        const EmuDesc& e = ed[tr.di];
        const int nch = e.Kp / kChunk;
        for (int c = 0; c < nch && good; ++c)
          for (int hf = 0; hf < 2; ++hf, ++q) {
            const int s = q % kCStages, u = q / kCStages;
            if (q >= kCStages && !mbar_wait_ab(bar(3 + s), (u - 1) & 1, abort_flag, wait_ns)) {
              good = false;
              break;
            }
            mbar_expect_tx(bar(s), (unsigned)kCStage);
            const int64_t ablk = (int64_t)tr.rb * nch + c, bblk = (int64_t)tr.j * nch + c;
            for (int p = 0; p < ND; ++p)
              bulk_g2s(smem_u32(stageA(s) + p * kAHalf), Wd + e.adig + (ablk * ND + p) * 4096 + hf * 2048, kAHalf,
                       bar(s));
            bulk_g2s(smem_u32(stageB(s)), Wd + e.bdig + bblk * (1024 * ND) + hf * (512 * ND), ND * kBHalf, bar(s));
          }
      }
      if (!good) {
        *abort_flag = 1;
        set_status(status, CL_ERR_TIMEOUT, -8, t0);
      }
      if (*abort_flag)  // copies still in flight: the last stages, bounded
        for (int i = max(0, q - kCStages); i < q; ++i) mbar_wait(bar(i % kCStages), (i / kCStages) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      int q = 0, k = 0;
      bool good = true;
      // the last commit issued (it arrives once every earlier MMA of this
      // thread has completed): what a teardown after a timeout waits for
      uint32_t lc_bar = 0;
      unsigned lc_par = 0;
      bool has_lc = false;
      for (int t = t0; t < t1 && good && !*abort_flag; t += G) {
        const TileRef tr = tile_ref(gd, d0, d1, t);
        const int nch = ed[tr.di].Kp / kChunk;
        for (int c = 0; c < nch && good; ++c, ++k) {
          const int set = k & 1, uk = k >> 1;
          if (k >= 2 && !mbar_wait_ab(bar(8 + set), (uk - 1) & 1, abort_flag, wait_ns)) {
            good = false;
            break;
          }
          for (int hf = 0; hf < 2; ++hf, ++q) {
            const int s = q % kCStages, u = q / kCStages;
            if (!mbar_wait_ab(bar(s), u & 1, abort_flag, wait_ns)) {
              good = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(stageA(s)), b0 = smem_u32(stageB(s)), d = tmem + 256u * set;
#pragma unroll 1
            for (int p = 0; p < ND; ++p)
#pragma unroll
              for (int kb = 0; kb < 2; ++kb)
                umma_bf16(d + 32 * p, umma_desc(a0 + p * kAHalf + kb * 4096), umma_desc(b0 + kb * (ND * 1024)),
                          tc_idesc(ND, p), (hf | p | kb) != 0 ? 1u : 0u);
            umma_commit(bar(3 + s));
            lc_bar = bar(3 + s);
            lc_par = (unsigned)(u & 1);
            has_lc = true;
          }
          if (!good) break;
          umma_commit(bar(6 + set));
        }
      }
      if (!good) {
        *abort_flag = 1;
        set_status(status, CL_ERR_TIMEOUT, -9, t0);
      }
      if (*abort_flag && has_lc) mbar_wait(lc_bar, lc_par);  // MMAs in flight, a half chunk included
    }
    __syncwarp();
  } else {  // ---- fold and epilogue: group g owns complex columns CC g .. CC g + CC-1 of the tile
    constexpr int CR = 32 / NG, CC = CR / 2;  // real / complex columns of a group
    const int grp = (warp - 2) >> 2, q4 = warp & 3, rl = q4 * 32 + lane;
    int k = 0;
    bool stop = false;
    for (int t = t0; t < t1 && !stop; t += G) {
      const TileRef tr = tile_ref(gd, d0, d1, t);
      const GemmDesc g = gd[tr.di];
      const EmuDesc e = ed[tr.di];
      const int nch = e.Kp / kChunk;
      const int row = tr.rb * 128 + rl, c8 = tr.j * kTileCx + CC * grp;
      // row / column maxima of the chunk exponents (column jj = lane jj of each warp)
      int Rm = -4000, Sc = -4000;
      for (int c = 0; c < nch; ++c) {
        Rm = max(Rm, Id[e.aexp + (int64_t)c * e.Mp + row]);
        if (lane < CC) Sc = max(Sc, Id[e.bexp + (int64_t)c * e.Np + c8 + lane]);
      }
      int ra = nch > 0 ? Id[e.aexp + row] : 0;
      int cb = (lane < CC && nch > 0) ? Id[e.bexp + c8 + lane] : 0;
      float h[CR], mi[CR], lo[CR];
#pragma unroll
      for (int i = 0; i < CR; ++i) h[i] = mi[i] = lo[i] = 0.f;
      for (int c = 0; c < nch; ++c, ++k) {
        __syncwarp();
        const int rsc = ra - Rm - 16, csc = cb - Sc;
        if (c + 1 < nch) {
          ra = Id[e.aexp + (int64_t)(c + 1) * e.Mp + row];
          if (lane < CC) cb = Id[e.bexp + (int64_t)(c + 1) * e.Np + c8 + lane];
        }
        float sc[CC];  // 2^{(e_i - R_i) + (f_n - S_n) - 16}
#pragma unroll
        for (int jj = 0; jj < CC; ++jj) sc[jj] = pow2f(rsc + __shfl_sync(0xffffffffu, csc, jj));
        const int set = k & 1, uk = k >> 1;
        const bool got = mbar_wait_ab(bar(6 + set), uk & 1, abort_flag, wait_ns);
        if (!__all_sync(0xffffffffu, got)) {
          if (!*abort_flag) set_status(status, CL_ERR_TIMEOUT, -10, t0);
          *abort_flag = 1;
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + 256u * set + CR * grp;
#pragma unroll
        for (int b4 = 0; b4 < 2; ++b4) {  // levels 0-3, then 4 .. ND-1
          constexpr int N1 = ND < 4 ? ND : 4, N2 = ND - N1, E2 = ND >= 8 ? 1 : 0;
          const int L0 = 4 * b4, nl = b4 ? N2 : N1;
          if (nl == 0) continue;
          uint32_t v[4][CR];
#pragma unroll
          for (int l = 0; l < 4; ++l)
            if (l < nl) tmem_ld_issue(ta + 32 * (L0 + l), v[l]);
          tmem_ld_wait();
          if (b4 || N2 == 0) {
            tc_fence_before();
            mbar_arrive(bar(8 + set));  // accumulator set drained
          }
          if (b4) {  // levels 4 .. ND-1 (<= 2^-32 of the leading level): with 8 digits
                     // level 4 by an error-free addition of its own, the rest summed in
                     // FP32 and added by one more
#pragma unroll
            for (int i = 0; i < CR; ++i) {
              const float c = sc[i >> 1];
              float s2, e2;
              if (E2) {
                two_sum(mi[i], __uint_as_float(v[0][i]) * (c * 0x1p-32f), s2, e2);
                mi[i] = s2;
                lo[i] += e2;
              }
              float x = __uint_as_float(v[E2][i]) * (c * __int_as_float((127 - 32 - 8 * E2) << 23));
#pragma unroll
              for (int l = E2 + 1; l < 4; ++l)
                if (l < nl) x = fmaf(__uint_as_float(v[l][i]), c * __int_as_float((127 - 32 - 8 * l) << 23), x);
              two_sum(mi[i], x, s2, e2);
              mi[i] = s2;
              lo[i] += e2;
            }
          } else {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              if (l >= nl) continue;
              const float cL = __int_as_float((127 - 8 * l) << 23);  // 2^{-8L}
#pragma unroll
              for (int i = 0; i < CR; ++i) {
                const float x = __uint_as_float(v[l][i]) * (sc[i >> 1] * cL);
                float s1, e1, s2, e2;
                if (l < 2) {
                  two_sum(h[i], x, s1, e1);
                  h[i] = s1;
                  two_sum(mi[i], e1, s2, e2);
                } else {
                  two_sum(mi[i], x, s2, e2);
                }
                mi[i] = s2;
                lo[i] += e2;
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < CR; ++i) {
          float s1, e1, s2, e2;
          two_sum(h[i], mi[i], s1, e1);
          two_sum(e1, lo[i], s2, e2);
          h[i] = s1;
          mi[i] = s2;
          lo[i] = e2;
        }
      }
      if (stop) break;
      // epilogue of the tile: value = (h + mi + lo) 2^{R_i + S_n}; C = beta C -/+ value.
      // Column maxima from lanes 0-7, shuffled while every lane is present.
      int sx[CC];
#pragma unroll
      for (int jj = 0; jj < CC; ++jj) sx[jj] = __shfl_sync(0xffffffffu, Sc, jj);
      if (row >= g.M || g.rmask.hit(row)) continue;
      const bool ctr = (g.trans & 4) != 0;  // C stored transposed: column stride ldc
      const int64_t cs = ctr ? g.ldc : 1;
      double2* crow = arena + blockIdx.y * stride + g.c + (ctr ? (int64_t)row : (int64_t)row * g.ldc) + c8 * cs;
      const bool neg = g.neg != 0;
      double2 cv[CC];
      if (g.beta) {
#pragma unroll
        for (int jj = 0; jj < CC; ++jj) cv[jj] = c8 + jj < g.N ? crow[jj * cs] : make_double2(0, 0);
      }
#pragma unroll
      for (int jj = 0; jj < CC; ++jj) {
        const int cc = c8 + jj;
        const int ex = Rm + sx[jj];
        if (cc >= g.N || g.cmask.hit(cc)) continue;
        double vv[2];
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const int i = 2 * jj + part;
          float s1, e1;
          two_sum(h[i], mi[i], s1, e1);
          vv[part] = f2d_scaled(s1, ex, neg) + f2d_scaled(e1 + lo[i], ex, neg);
        }
        double2 v = make_double2(vv[0], vv[1]);
        if (g.beta) v = cadd(v, cv[jj]);
        crow[jj * cs] = v;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPCols) : "memory");
  }
}

}  // namespace

// opt the GEMM kernels in to > 48 KB of dynamic shared memory on the current
// device (done when a plan is set up, outside any stream capture)
template <int ND>
cudaError_t emu_prepare_nd() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_emu_chunked<kChunkedGroups, ND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c_smem_bytes(ND));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_emu_persist<2, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)p_smem_bytes(ND));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gemm_emu_persist<4, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)p_smem_bytes(ND));
}
cudaError_t emu_prepare() {
  cudaError_t e = emu_prepare_nd<3>();
  if (e == cudaSuccess) e = emu_prepare_nd<7>();
  if (e == cudaSuccess) e = emu_prepare_nd<8>();
  return e;
}

// fold groups of the persistent digit GEMM: four (576 threads, 96 registers)
// unless CLSELINV_FOLD_GROUPS=2 (measured at 8^3x4: 63.0 -> 66.4 evals/s,
// batch 64 77.5 -> 85.4; 12^3x6 0.477 -> 0.417 s)
int fold_groups() {
  static const int ng = [] {
    const char* v = std::getenv("CLSELINV_FOLD_GROUPS");
    return v && v[0] == '2' ? 2 : 4;
  }();
  return ng;
}

template <int ND>
cudaError_t launch_emu_nd(const GemmDesc* gd, const EmuDesc* ed, int d0, int d1, int items, int blocks, int batch,
                          double2* arena, int64_t stride, unsigned* words, int* ints, int64_t wstride,
                          int64_t istride, int* status, bool single_chunk, int max_ctas, cudaStream_t st,
                          LaunchOpt lo, unsigned long long wait_ns) {
  const dim3 gs((unsigned)((items + 7) / 8), (unsigned)batch);
  cudaError_t e = launch_k(k_emu_split<ND>, gs, dim3(256), 0, st, lo, gd, ed, d0, d1, (const double2*)arena, stride,
                           words, ints, wstride, istride, items, status);
  if (e != cudaSuccess) return e;
  const LaunchOpt lg{lo.prio, pdl_enabled()};  // follows the split pass in the same stream
  const dim3 gp((unsigned)std::min(blocks, std::max(max_ctas, 1)), (unsigned)batch);
  if (single_chunk)  // blocks = output tiles of the launch; persistent CTAs over ranges of tiles
    return fold_groups() == 4
               ? launch_k(k_gemm_emu_persist<4, ND>, gp, dim3(64 + 128 * 4), p_smem_bytes(ND), st, lg, gd, ed, d0,
                          d1, blocks, arena, stride, (const unsigned*)words, (const int*)ints, wstride, istride, status,
                          wait_ns)
               : launch_k(k_gemm_emu_persist<2, ND>, gp, dim3(64 + 128 * 2), p_smem_bytes(ND), st, lg, gd, ed, d0,
                          d1, blocks, arena, stride, (const unsigned*)words, (const int*)ints, wstride, istride,
                          status, wait_ns);
  return launch_k(k_gemm_emu_chunked<kChunkedGroups, ND>, gp, dim3(64 + 128 * kChunkedGroups), c_smem_bytes(ND), st,
                  lg, gd, ed, d0, d1, blocks, arena, stride, (const unsigned*)words, (const int*)ints, wstride,
                  istride, status, wait_ns);
}

cudaError_t launch_emu(const GemmDesc* gd, const EmuDesc* ed, int d0, int d1, int items, int blocks, int batch,
                       double2* arena, int64_t stride, unsigned* words, int* ints, int64_t wstride, int64_t istride,
                       int* status, bool single_chunk, int max_ctas, int ndig, cudaStream_t st, LaunchOpt lo,
                       unsigned long long wait_ns) {
  switch (ndig) {
    case 3:
      return launch_emu_nd<3>(gd, ed, d0, d1, items, blocks, batch, arena, stride, words, ints, wstride, istride,
                              status, single_chunk, max_ctas, st, lo, wait_ns);
    case 7:
      return launch_emu_nd<7>(gd, ed, d0, d1, items, blocks, batch, arena, stride, words, ints, wstride, istride,
                              status, single_chunk, max_ctas, st, lo, wait_ns);
    case 8:
      return launch_emu_nd<8>(gd, ed, d0, d1, items, blocks, batch, arena, stride, words, ints, wstride, istride,
                              status, single_chunk, max_ctas, st, lo, wait_ns);
    default:
      return cudaErrorInvalidValue;
  }
}

// A persistent bulk CTA (576 threads x 96 registers) leaves too few
// registers on its SM for a panel-inverse CTA, so a bulk launch over every SM
// would hold the next panel until the whole bulk update ends: bulk launches
// (stream 1) leave p.chain_sms SMs to the panel chain.
cudaError_t launch_gemm_emu(const Plan& p, const Op& op, double2* arena, cudaStream_t st) {
  const int items = p.emu[op.d1 - 1].it0 + p.emu[op.d1 - 1].items;
  const int ctas = op.stream ? std::max(1, p.num_sms - p.chain_sms) : p.num_sms;
  return launch_emu(p.d_gemm, p.d_emu, op.d0, op.d1, items, op.blocks, p.fbatch, arena, p.arena_elems,
                    p.d_emu_words, p.d_emu_ints, p.emu_words, p.emu_ints, p.d_status, op.single_chunk, ctas, op.ndig,
                    st, op_launch(p, op), p.wait_ns);
}

}  // namespace cl

// ---------------------------------------------------------------------------
// Stand-alone FP64-accurate complex GEMM through the same kernels.
namespace {

constexpr int kZgemmDigits = 7;  // the stand-alone GEMM: an FP64 GEMM's accuracy

struct ZgemmLayout {
  cl::GemmDesc g;
  cl::EmuDesc e;
  int blocks;
  size_t desc_off, words_off, ints_off, total;
};

bool zgemm_layout(int M, int N, int K, ZgemmLayout& z) {
  if (M < 1 || N < 1 || K < 1) return false;
  std::memset(&z, 0, sizeof(z));
  cl::EmuDesc& e = z.e;
  e.Mp = (M + 127) / 128 * 128;
  e.Np = (N + 31) / 32 * 32;
  e.Kp = (K + 31) / 32 * 32;
  const int64_t nch = e.Kp / 32;
  e.adig = 0;
  e.bdig = ((int64_t)kZgemmDigits * e.Mp * e.Kp + 63) / 64 * 64;
  const int64_t words = e.bdig + ((int64_t)kZgemmDigits * 2 * e.Np * e.Kp + 63) / 64 * 64;
  e.aexp = 0;
  e.bexp = nch * e.Mp;
  const int64_t ints = e.bexp + nch * e.Np;
  e.it0 = 0;
  e.items = (int)(e.Mp * nch + e.Np * nch);
  z.blocks = (e.Mp / 128) * (e.Np / 16);
  z.desc_off = 0;
  z.words_off = 1024;
  z.ints_off = z.words_off + (size_t)words * 4;
  z.total = (z.ints_off + (size_t)ints * 4 + 255) / 256 * 256;
  return true;
}

}  // namespace

extern "C" int cl_zgemm_emu_workspace(int M, int N, int K, size_t* bytes) {
  ZgemmLayout z;
  if (!bytes || !zgemm_layout(M, N, K, z)) return CL_ERR_INVALID_ARG;
  *bytes = z.total;
  return CL_OK;
}

extern "C" int cl_zgemm_emu(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                            int beta, int neg, void* work, size_t work_bytes, int* status, cudaStream_t stream) {
  ZgemmLayout z;
  if (!zgemm_layout(M, N, K, z) || !A || !B || !C || !work || !status || lda < K || ldb < N || ldc < N)
    return CL_ERR_INVALID_ARG;
  if (work_bytes < z.total) return CL_ERR_INVALID_ARG;
  const uintptr_t ua = (uintptr_t)A, ub = (uintptr_t)B, uc = (uintptr_t)C;
  if ((ua | ub | uc) & 15u || (uintptr_t)work & 255u) return CL_ERR_INVALID_ARG;
  // operands addressed as offsets (in complex elements) from A
  z.g.a = 0;
  z.g.b = ((int64_t)ub - (int64_t)ua) / 16;
  z.g.c = ((int64_t)uc - (int64_t)ua) / 16;
  z.g.lda = lda;
  z.g.ldb = ldb;
  z.g.ldc = ldc;
  z.g.M = M;
  z.g.N = N;
  z.g.K = K;
  z.g.neg = neg ? 1 : 0;
  z.g.beta = beta ? 1 : 0;
  z.g.blk0 = 0;
  z.g.tilesN = z.e.Np / 16;
  static thread_local int prepared_dev = -1, sms = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
  if (prepared_dev != dev) {
    if (cl::emu_prepare() != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return CL_ERR_CUDA;
    prepared_dev = dev;
  }
  unsigned char* wb = static_cast<unsigned char*>(work);
  unsigned char host[256];
  std::memcpy(host, &z.g, sizeof(z.g));
  std::memcpy(host + 128, &z.e, sizeof(z.e));
  static_assert(sizeof(cl::GemmDesc) <= 128 && sizeof(cl::EmuDesc) <= 128, "descriptor block");
  cudaError_t e = cudaMemcpyAsync(wb, host, 256, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return CL_ERR_CUDA;
  e = cl::launch_emu(reinterpret_cast<const cl::GemmDesc*>(wb), reinterpret_cast<const cl::EmuDesc*>(wb + 128), 0, 1,
                     z.e.items, z.blocks, 1, reinterpret_cast<double2*>(const_cast<double*>(A)), 0,
                     reinterpret_cast<unsigned*>(wb + z.words_off), reinterpret_cast<int*>(wb + z.ints_off), 0, 0,
                     status, z.e.Kp == 32, sms, kZgemmDigits, stream, cl::LaunchOpt{}, cl::kDefaultWaitNs);
  return e == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}
