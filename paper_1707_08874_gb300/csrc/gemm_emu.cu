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

}  // namespace

size_t emu_smem_bytes() { return kEmuSmemBytes; }

// opt the GEMM kernel in to > 48 KB of dynamic shared memory on the current
// device (done when a plan is set up, outside any stream capture)
cudaError_t emu_prepare() {
  return cudaFuncSetAttribute(k_gemm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEmuSmemBytes);
}

cudaError_t launch_gemm_emu(const Plan& p, const Op& op, double2* arena, cudaStream_t st) {
  const int items = p.emu[op.d1 - 1].it0 + p.emu[op.d1 - 1].items;
  const dim3 gs((unsigned)((items + 7) / 8), (unsigned)p.batch);
  k_emu_split<<<gs, 256, 0, st>>>(p.d_gemm, p.d_emu, op.d0, op.d1, arena, p.arena_elems, p.d_emu_words, p.d_emu_ints,
                                  p.emu_words, p.emu_ints, items);
  const dim3 gg((unsigned)op.blocks, (unsigned)p.batch);
  k_gemm_emu<<<gg, 256, kEmuSmemBytes, st>>>(p.d_gemm, p.d_emu, op.d0, op.d1, arena, p.arena_elems, p.d_emu_words,
                                             p.d_emu_ints, p.emu_words, p.emu_ints);
  return cudaGetLastError();
}

}  // namespace cl
