// FP64-accurate complex GEMM on the BF16 tensor cores (precision CL_FP64_EMU).
//
// GB300's FP64 pipe delivers ~1.1 TFLOP/s, its BF16 tensor pipe ~590 TFLOP/s
// through mma.sync.  Each FP64 operand is written exactly as
//   a = sign * 2^e * sum_{p=1..7} d_p 2^{-8p} + (truncation < 2^{e-56}),
// with integer digits 0 <= d_p <= 255 (exact in BF16) and one exponent e per
// row (A) or column (B) and per chunk of 32 complex k.  The product is the sum
// over digit pairs p + q <= 8 (28 BF16 products) of integer dot products: each
// one is exact in the FP32 accumulator for the leading levels (sums < 2^24) and
// rounded below FP64 resolution for the others.  Level sums are scaled by
// powers of two and accumulated across chunks in triple-float (three FP32
// words, error-free two-sums), relative to the largest row / column exponent;
// FP64 arithmetic appears only in the epilogue (two additions per output).  Accuracy equals an FP64 GEMM
// to within a small factor (numpy emulation of the same digits and roundings:
// normwise relative error 4e-16 - 1.1e-15 against 5e-16 - 1e-15 for FP64).
//
// Complex products are one real product of twice the size, as in the FP64
// kernel: A is the real M x 2K matrix of interleaved pairs; B is expanded into
// [[br, bi], [-bi, br]] blocks when its fragment is loaded from shared memory.
#include <cstring>

#include "kernels.cuh"

namespace cl {
namespace {

constexpr int kDig = 7;       // base-256 digits per operand
constexpr int kLevels = 7;    // digit pairs p + q <= 6 (0-based) -> 28 products
constexpr int kChunk = 32;    // complex k per exponent chunk (64 real k)
constexpr int kStrideW = 36;  // shared-memory row stride in 32-bit words (32 + 4 pad)

__device__ __forceinline__ int exp_of(double v) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? -2000 : E - 1023;  // zero / subnormal count as absent
}

// BF16 bit patterns of the 7 digits of |v| 2^{-e} (< 1), truncated, with v's sign
__device__ __forceinline__ void digits(double v, int e, unsigned short (&d)[kDig]) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned short sgn = b < 0 ? 0x8000u : 0u;
  unsigned long long X = 0;
  if (E != 0 && E != 0x7FF) {
    const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (E - 1023) + 4 - e;  // X = m 2^sh = |v| 2^{56-e}; sh <= 3
    if (sh >= 0) X = m << sh;
    else if (sh > -64) X = m >> (-sh);
  }
#pragma unroll
  for (int p = 0; p < kDig; ++p) {
    const unsigned dg = (unsigned)(X >> (48 - 8 * p)) & 0xFFu;
    d[p] = dg ? (unsigned short)((__float_as_uint((float)dg) >> 16) | sgn) : (unsigned short)0;
  }
}

// Split pass: one warp per item.  A items (row, chunk): lanes take the 32
// complex k of the chunk; digits go to A[p][row][k] as (re, im) BF16 pairs.
// B items (column n, chunk): lanes take the chunk's 32 k; the real embedding
// of b = br + i bi is written directly, k-contiguous, as two rows of B'^T:
//   row 2n   : (br, -bi)   (real column 2n of [[br, bi], [-bi, br]] per k)
//   row 2n+1 : (bi,  br)
// so the GEMM loads both operands with ldmatrix and no per-element work.
// Padding (rows >= M, columns >= N, k >= K) gets zero digits.
// Tiled layout (tensor-core path): every (digit, 128-row block, chunk) of A
// and every (digit, 64-real-column block, chunk) of B' is one contiguous tile
// in the order the tensor core reads shared memory without swizzling: 16-k
// slabs, inside a slab 8-row groups of two 8 x 8 core matrices (k 0-7, 8-15),
// each core matrix 8 rows of 16 bytes.  A tile is then one bulk copy.
__device__ __forceinline__ int64_t a_tile_word(const EmuDesc& e, int nch, int p, int row, int c, int lane) {
  const int64_t tile = ((int64_t)p * (e.Mp / 128) + row / 128) * nch + c;
  const int r = row & 127;
  return e.adig + tile * 4096 + (lane >> 3) * 1024 + (r >> 3) * 64 + ((lane >> 2) & 1) * 32 + (r & 7) * 4 + (lane & 3);
}
__device__ __forceinline__ int64_t b_tile_word(const EmuDesc& e, int nch, int q, int nreal, int c, int lane) {
  const int64_t tile = ((int64_t)q * (e.Np / 32) + nreal / 64) * nch + c;
  const int r = nreal & 63;
  return e.bdig + tile * 2048 + (lane >> 3) * 512 + (r >> 3) * 64 + ((lane >> 2) & 1) * 32 + (r & 7) * 4 + (lane & 3);
}

template <bool kTiled>
__global__ void __launch_bounds__(256) k_emu_split(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed,
                                                   int d0, int d1, const double2* __restrict__ arena,
                                                   int64_t stride, unsigned* __restrict__ words,
                                                   int* __restrict__ ints, int64_t wstride, int64_t istride,
                                                   int total) {
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
    if (line < g.M && k < g.K) v = base[g.a + (int64_t)line * g.lda + k];
  } else {
    if (line < g.N && k < g.K) v = base[g.b + (int64_t)k * g.ldb + line];
  }
  int ex = max(exp_of(v.x), exp_of(v.y));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
  const int ee = ex + 1;
  unsigned short dr[kDig], di[kDig];
  digits(v.x, ee, dr);
  digits(v.y, ee, di);
  if (kTiled) {
    if (isA) {
      if (lane == 0) I[e.aexp + (int64_t)c * e.Mp + line] = ee;
#pragma unroll
      for (int p = 0; p < kDig; ++p) W[a_tile_word(e, nch, p, line, c, lane)] = (unsigned)dr[p] | ((unsigned)di[p] << 16);
    } else {
      if (lane == 0) I[e.bexp + (int64_t)c * e.Np + line] = ee;
#pragma unroll
      for (int p = 0; p < kDig; ++p) {
        W[b_tile_word(e, nch, p, 2 * line, c, lane)] =
            (unsigned)dr[p] | ((unsigned)(di[p] ^ (di[p] ? 0x8000u : 0u)) << 16);
        W[b_tile_word(e, nch, p, 2 * line + 1, c, lane)] = (unsigned)di[p] | ((unsigned)dr[p] << 16);
      }
    }
    return;
  }
  if (isA) {
    if (lane == 0) I[e.aexp + (int64_t)c * e.Mp + line] = ee;
    unsigned* dst = W + e.adig + (int64_t)line * e.Kp + k;
#pragma unroll
    for (int p = 0; p < kDig; ++p) dst[(int64_t)p * e.Mp * e.Kp] = (unsigned)dr[p] | ((unsigned)di[p] << 16);
  } else {
    if (lane == 0) I[e.bexp + (int64_t)c * e.Np + line] = ee;
    unsigned* dst0 = W + e.bdig + (int64_t)(2 * line) * e.Kp + k;
    unsigned* dst1 = dst0 + e.Kp;
    const int64_t plane = (int64_t)2 * e.Np * e.Kp;
#pragma unroll
    for (int p = 0; p < kDig; ++p) {
      dst0[p * plane] = (unsigned)dr[p] | ((unsigned)(di[p] ^ (di[p] ? 0x8000u : 0u)) << 16);
      dst1[p * plane] = (unsigned)di[p] | ((unsigned)dr[p] << 16);
    }
  }
}

__device__ __forceinline__ void bmma(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                     unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
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

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void ldsm4(unsigned (&r)[4], const unsigned* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

constexpr int kEmuTM = 128;                        // rows per CTA
constexpr int kSmemA = kDig * kEmuTM * kStrideW;   // words
constexpr int kSmemB = kDig * 64 * kStrideW;       // 64 real columns (32 complex)
constexpr size_t kEmuSmemBytes = (size_t)(kSmemA + kSmemB) * 4 + (kEmuTM + 32) * 2 * sizeof(int);

// 256 threads = 4 x 2 warps; each warp owns 32 rows x 32 real columns
// (2 x 4 MMA tiles of 16 x 8); CTA tile 128 rows x 32 complex columns.
__global__ void __launch_bounds__(256, 1) k_gemm_emu(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed,
                                                     int d0, int d1, double2* __restrict__ arena, int64_t stride,
                                                     const unsigned* __restrict__ words, const int* __restrict__ ints,
                                                     int64_t wstride, int64_t istride) {
  extern __shared__ __align__(16) unsigned smem[];
  unsigned* As = smem;
  unsigned* Bs = smem + kSmemA;
  int* rsc = reinterpret_cast<int*>(Bs + kSmemB);  // [128] chunk exponent minus the row maximum
  int* csc = rsc + kEmuTM;                         // [32]  same for the complex columns
  int* Rm = csc + 32;                              // [128] row maxima
  int* Sm = Rm + kEmuTM;                           // [32]  column maxima

  const int di = find_desc(gd, d0, d1, blockIdx.x);
  const GemmDesc g = gd[di];
  const EmuDesc e = ed[di];
  const int t = blockIdx.x - g.blk0;
  const int row0 = (t / g.tilesN) * kEmuTM, col0 = (t % g.tilesN) * kTileN;
  const unsigned* Wd = words + blockIdx.y * wstride;
  const int* Id = ints + blockIdx.y * istride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 16;  // row / complex column offsets of the warp
  const int nch = e.Kp / kChunk;

  if (tid < kEmuTM) {
    int m = -4000;
    for (int c = 0; c < nch; ++c) m = max(m, Id[e.aexp + (int64_t)c * e.Mp + row0 + tid]);
    Rm[tid] = m;
  } else if (tid < kEmuTM + 32) {
    int m = -4000;
    for (int c = 0; c < nch; ++c) m = max(m, Id[e.bexp + (int64_t)c * e.Np + col0 + tid - kEmuTM]);
    Sm[tid - kEmuTM] = m;
  }

  float h[2][4][4], mi[2][4][4], lo[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) h[i][j][r] = mi[i][j][r] = lo[i][j][r] = 0.f;

  // ldmatrix lane addressing: A rows (lane & 15), k half (lane >> 4);
  // B' rows n_r = 8j + (lane & 7) + 8 ((lane >> 4) & 1), k half ((lane >> 3) & 1)
  const int a_row = lane & 15, a_kw = (lane >> 4) * 4;
  const int b_row = (lane & 7) + ((lane >> 4) & 1) * 8, b_kw = ((lane >> 3) & 1) * 4;

  for (int c = 0; c < nch; ++c) {
    for (int q = tid; q < kDig * kEmuTM * 8; q += 256) {
      const int p = q / (kEmuTM * 8), r = (q / 8) % kEmuTM, piece = q % 8;
      cp16(As + (p * kEmuTM + r) * kStrideW + piece * 4,
           Wd + e.adig + (int64_t)p * e.Mp * e.Kp + (int64_t)(row0 + r) * e.Kp + c * kChunk + piece * 4);
    }
    for (int q = tid; q < kDig * 64 * 8; q += 256) {
      const int p = q / (64 * 8), r = (q / 8) % 64, piece = q % 8;
      cp16(Bs + (p * 64 + r) * kStrideW + piece * 4,
           Wd + e.bdig + (int64_t)p * 2 * e.Np * e.Kp + (int64_t)(2 * col0 + r) * e.Kp + c * kChunk + piece * 4);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    __syncthreads();  // row / column maxima visible before the scale factors
    if (tid < kEmuTM) rsc[tid] = Id[e.aexp + (int64_t)c * e.Mp + row0 + tid] - Rm[tid];
    else if (tid < kEmuTM + 32) csc[tid - kEmuTM] = Id[e.bexp + (int64_t)c * e.Np + col0 + tid - kEmuTM] - Sm[tid - kEmuTM];
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();

    float scl[2][4][2];  // 2^{(e_i - R_i) + (f_n - S_n) - 16} per owned (row pair, column)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
          scl[i][j][rr] = pow2f(rsc[wm + 16 * i + gq + 8 * rr] + csc[wn + 4 * j + tq] - 16);

#pragma unroll 1
    for (int L = 0; L < kLevels; ++L) {
      float acc[2][4][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
#pragma unroll 2
      for (int p = 0; p <= L; ++p) {
        const unsigned* Ap = As + (p * kEmuTM + wm + a_row) * kStrideW + a_kw;
        const unsigned* Bq = Bs + ((L - p) * 64 + 2 * wn + b_row) * kStrideW + b_kw;
#pragma unroll
        for (int ks = 0; ks < kChunk / 8; ++ks) {
          unsigned a[2][4], b[4][2];
          ldsm4(a[0], Ap + ks * 8);
          ldsm4(a[1], Ap + 16 * kStrideW + ks * 8);
          unsigned t4[4];
          ldsm4(t4, Bq + ks * 8);
          b[0][0] = t4[0]; b[0][1] = t4[1]; b[1][0] = t4[2]; b[1][1] = t4[3];
          ldsm4(t4, Bq + 16 * kStrideW + ks * 8);
          b[2][0] = t4[0]; b[2][1] = t4[1]; b[3][0] = t4[2]; b[3][1] = t4[3];
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) bmma(acc[i][j], a[i][0], a[i][1], a[i][2], a[i][3], b[j][0], b[j][1]);
        }
      }
      // fold: levels 0, 1 into (h, mi, lo); levels >= 2 are below 2^-32 of the
      // leading level and go straight into (mi, lo)
      const float cL = __int_as_float((127 - 8 * L) << 23);  // 2^{-8L}
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float x = acc[i][j][r] * (scl[i][j][r >> 1] * cL);
            float s, e1, s2, e2;
            if (L < 2) {
              two_sum(h[i][j][r], x, s, e1);
              h[i][j][r] = s;
              two_sum(mi[i][j][r], e1, s2, e2);
            } else {
              two_sum(mi[i][j][r], x, s2, e2);
            }
            mi[i][j][r] = s2;
            lo[i][j][r] += e2;
          }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float s, e1, s2, e2;
          two_sum(h[i][j][r], mi[i][j][r], s, e1);
          two_sum(e1, lo[i][j][r], s2, e2);
          h[i][j][r] = s;
          mi[i][j][r] = s2;
          lo[i][j][r] = e2;
        }
    __syncthreads();
  }

  // epilogue: value = (h + mi + lo) 2^{R_i + S_n}; C = beta C -/+ value.
  // Two exact float -> double conversions by bit manipulation, then at most
  // two FP64 additions per real output.
  double2* C = arena + blockIdx.y * stride + g.c;
  const bool neg = g.neg != 0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int rl = wm + 16 * i + gq + rr * 8, cl = wn + 4 * j + tq;
        const int r = row0 + rl, cc = col0 + cl;
        if (r >= g.M || cc >= g.N) continue;
        if (g.rmask.hit(r) || g.cmask.hit(cc)) continue;
        const int ex = Rm[rl] + Sm[cl];
        double vv[2];
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const int q = 2 * rr + part;
          float s, e1;
          two_sum(h[i][j][q], mi[i][j][q], s, e1);
          vv[part] = f2d_scaled(s, ex, neg) + f2d_scaled(e1 + lo[i][j][q], ex, neg);
        }
        double2 v = make_double2(vv[0], vv[1]);
        double2* pc = C + (int64_t)r * g.ldc + cc;
        if (g.beta) v = cadd(v, *pc);
        *pc = v;
      }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) digit GEMM.  Same digits, levels, fold and epilogue
// as k_gemm_emu; the 28 digit products of a chunk are 112 asynchronous
// 128 x 64 x 16 BF16 MMAs issued by one thread, accumulated in tensor memory
// (one 64-column FP32 accumulator per level, 448 of the SM's 512 columns),
// with operands brought into shared memory by bulk copies of the pre-tiled
// digit planes.  CTA tile 128 rows x 32 complex columns, 256 threads: thread
// (w, l) folds row 32 (w % 4) + l, real columns 32 (w / 4) .. + 31.
// Every wait on an mbarrier gives up after a bounded time, records
// CL_ERR_TIMEOUT and leaves through the normal teardown (TMEM freed).
constexpr int kTcA = 4096 * 4;  // bytes of one A digit tile (128 rows x 64 real k)
constexpr int kTcB = 2048 * 4;  // bytes of one B' digit tile (64 real columns x 64 real k)
constexpr uint32_t kTcCols = 512;
constexpr int kTcCtl = 2048;    // control block: mbarriers, TMEM address, exponents
constexpr size_t kTcSmemBytes = (size_t)kDig * (kTcA + kTcB) + kTcCtl;
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr unsigned long long kWaitNs = 500000000ull;  // 0.5 s

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
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, unsigned long long ad, unsigned long long bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(256, 1)
    k_gemm_emu_tc(const GemmDesc* __restrict__ gd, const EmuDesc* __restrict__ ed, int d0, int d1,
                  double2* __restrict__ arena, int64_t stride, const unsigned* __restrict__ words,
                  const int* __restrict__ ints, int64_t wstride, int64_t istride, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;
  unsigned char* sB = smem_tc + kDig * kTcA;
  unsigned char* ctl = sB + kDig * kTcB;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ctl);  // [0] operands landed, [1] MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 16);
  int* abort_flag = reinterpret_cast<int*>(ctl + 20);
  int* Rm = reinterpret_cast<int*>(ctl + 64);  // [128] row maxima of the chunk exponents
  int* Sm = Rm + 128;                          // [32]  column maxima
  int* rsc = Sm + 32;                          // [128] chunk exponent minus the row maximum
  int* csc = rsc + 128;                        // [32]  same for the columns

  const int di = find_desc(gd, d0, d1, blockIdx.x);
  const GemmDesc g = gd[di];
  const EmuDesc e = ed[di];
  const int t = blockIdx.x - g.blk0;
  const int rb = t / g.tilesN, nb = t % g.tilesN;
  const int row0 = rb * 128, col0 = nb * 32;
  const unsigned* Wd = words + blockIdx.y * wstride;
  const int* Id = ints + blockIdx.y * istride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nch = e.Kp / kChunk;
  const uint32_t s_full = smem_u32(&bars[0]), s_done = smem_u32(&bars[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    mbar_init(s_full, 1);
    mbar_init(s_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 128) {
    int m = -4000;
    for (int c = 0; c < nch; ++c) m = max(m, Id[e.aexp + (int64_t)c * e.Mp + row0 + tid]);
    Rm[tid] = m;
  } else if (tid < 160) {
    int m = -4000;
    for (int c = 0; c < nch; ++c) m = max(m, Id[e.bexp + (int64_t)c * e.Np + col0 + tid - 128]);
    Sm[tid - 128] = m;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto issue_copies = [&](int c) {
    mbar_expect_tx(s_full, (unsigned)(kDig * (kTcA + kTcB)));
#pragma unroll 1
    for (int p = 0; p < kDig; ++p) {
      const unsigned* srcA = Wd + e.adig + (((int64_t)p * (e.Mp / 128) + rb) * nch + c) * 4096;
      const unsigned* srcB = Wd + e.bdig + (((int64_t)p * (e.Np / 32) + nb) * nch + c) * 2048;
      bulk_g2s(smem_u32(sA + p * kTcA), srcA, kTcA, s_full);
      bulk_g2s(smem_u32(sB + p * kTcB), srcB, kTcB, s_full);
    }
  };

  const int qd = warp & 3, hc = warp >> 2;
  const int rl = qd * 32 + lane;  // tile row of this thread
  float h[32], mi[32], lo[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) h[i] = mi[i] = lo[i] = 0.f;

  if (tid == 0 && nch > 0) issue_copies(0);  // K = 0: no operands, C = beta C
  bool ok = true;
#pragma unroll 1
  for (int c = 0; c < nch; ++c) {
    if (tid < 128) rsc[tid] = Id[e.aexp + (int64_t)c * e.Mp + row0 + tid] - Rm[tid];
    else if (tid < 160) csc[tid - 128] = Id[e.bexp + (int64_t)c * e.Np + col0 + tid - 128] - Sm[tid - 128];
    __syncthreads();
    if (tid == 0) {
      if (mbar_wait(s_full, c & 1)) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
        for (int L = 0; L < kLevels; ++L)
#pragma unroll 1
          for (int p = 0; p <= L; ++p)
#pragma unroll
            for (int kb = 0; kb < 4; ++kb)
              umma_bf16(tmem + 64 * L, umma_desc(a0 + p * kTcA + kb * 4096),
                        umma_desc(b0 + (L - p) * kTcB + kb * 2048), (p > 0 || kb > 0) ? 1u : 0u);
        umma_commit(s_done);
      } else {
        *abort_flag = 1;
        set_status(status, CL_ERR_TIMEOUT, -1, c);
        mbar_wait(s_full, c & 1);  // copies still in flight: wait once more
        mbar_arrive(s_done);       // no MMA issued: release the other threads
      }
    }
    const bool got = mbar_wait(s_done, c & 1);
    tc_fence_after();
    if (!got) set_status(status, CL_ERR_TIMEOUT, -2, c);
    if (__syncthreads_or(!got || *abort_flag)) {
      ok = false;
      if (tid == 0 && !*abort_flag) mbar_wait(s_done, c & 1);  // MMAs may still run: wait once more
      break;
    }
    if (tid == 0 && c + 1 < nch) issue_copies(c + 1);  // operands of chunk c consumed

    float sc[16];  // 2^{(e_i - R_i) + (f_n - S_n) - 16} for this row and the 16 complex columns
    const int rs = rsc[rl] - 16;
#pragma unroll
    for (int j = 0; j < 16; ++j) sc[j] = pow2f(rs + csc[hc * 16 + j]);
#pragma unroll 1
    for (int L = 0; L < kLevels; ++L) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + 64 * L + 32 * hc, v);
      const float cL = __int_as_float((127 - 8 * L) << 23);  // 2^{-8L}
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float x = __uint_as_float(v[i]) * (sc[i >> 1] * cL);
        float s, e1, s2, e2;
        if (L < 2) {
          two_sum(h[i], x, s, e1);
          h[i] = s;
          two_sum(mi[i], e1, s2, e2);
        } else {
          two_sum(mi[i], x, s2, e2);
        }
        mi[i] = s2;
        lo[i] += e2;
      }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float s, e1, s2, e2;
      two_sum(h[i], mi[i], s, e1);
      two_sum(e1, lo[i], s2, e2);
      h[i] = s;
      mi[i] = s2;
      lo[i] = e2;
    }
    tc_fence_before();
    __syncthreads();  // accumulators read: the next chunk's MMAs may overwrite them
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
  if (!ok) return;

  double2* C = arena + blockIdx.y * stride + g.c;
  const bool neg = g.neg != 0;
  const int r = row0 + rl;
  if (r >= g.M || g.rmask.hit(r)) return;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int cl = hc * 16 + j, cc = col0 + cl;
    if (cc >= g.N || g.cmask.hit(cc)) continue;
    const int ex = Rm[rl] + Sm[cl];
    double vv[2];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const int q = 2 * j + part;
      float s, e1;
      two_sum(h[q], mi[q], s, e1);
      vv[part] = f2d_scaled(s, ex, neg) + f2d_scaled(e1 + lo[q], ex, neg);
    }
    double2 v = make_double2(vv[0], vv[1]);
    double2* pc = C + (int64_t)r * g.ldc + cc;
    if (g.beta) v = cadd(v, *pc);
    *pc = v;
  }
}

}  // namespace

size_t emu_smem_bytes() { return kEmuSmemBytes; }

// opt the GEMM kernel in to > 48 KB of dynamic shared memory on the current
// device (done when a plan is set up, outside any stream capture)
cudaError_t emu_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEmuSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gemm_emu_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
}

cudaError_t launch_emu(const GemmDesc* gd, const EmuDesc* ed, int d0, int d1, int items, int blocks, int batch,
                       double2* arena, int64_t stride, unsigned* words, int* ints, int64_t wstride, int64_t istride,
                       int* status, bool tc, cudaStream_t st) {
  const dim3 gs((unsigned)((items + 7) / 8), (unsigned)batch);
  const dim3 gg((unsigned)blocks, (unsigned)batch);
  if (tc) {
    k_emu_split<true><<<gs, 256, 0, st>>>(gd, ed, d0, d1, arena, stride, words, ints, wstride, istride, items);
    k_gemm_emu_tc<<<gg, 256, kTcSmemBytes, st>>>(gd, ed, d0, d1, arena, stride, words, ints, wstride, istride,
                                                 status);
  } else {
    k_emu_split<false><<<gs, 256, 0, st>>>(gd, ed, d0, d1, arena, stride, words, ints, wstride, istride, items);
    k_gemm_emu<<<gg, 256, kEmuSmemBytes, st>>>(gd, ed, d0, d1, arena, stride, words, ints, wstride, istride);
  }
  return cudaGetLastError();
}

cudaError_t launch_gemm_emu(const Plan& p, const Op& op, double2* arena, cudaStream_t st) {
  const int items = p.emu[op.d1 - 1].it0 + p.emu[op.d1 - 1].items;
  return launch_emu(p.d_gemm, p.d_emu, op.d0, op.d1, items, op.blocks, p.batch, arena, p.arena_elems,
                    p.d_emu_words, p.d_emu_ints, p.emu_words, p.emu_ints, p.d_status, p.emu_tc, st);
}

}  // namespace cl

// ---------------------------------------------------------------------------
// Stand-alone FP64-accurate complex GEMM through the same kernels.
namespace {

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
  e.bdig = (7LL * e.Mp * e.Kp + 63) / 64 * 64;
  const int64_t words = e.bdig + (7LL * 2 * e.Np * e.Kp + 63) / 64 * 64;
  e.aexp = 0;
  e.bexp = nch * e.Mp;
  const int64_t ints = e.bexp + nch * e.Np;
  e.it0 = 0;
  e.items = (int)(e.Mp * nch + e.Np * nch);
  z.blocks = (e.Mp / 128) * (e.Np / 32);
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
  z.g.tilesN = z.e.Np / 32;
  static thread_local int prepared_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
  if (prepared_dev != dev) {
    if (cl::emu_prepare() != cudaSuccess) return CL_ERR_CUDA;
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
                     status, true, stream);
  return e == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}
