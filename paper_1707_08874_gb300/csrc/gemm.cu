// Batched complex GEMM of the front updates, C = beta*C -/+ A*B, one launch
// per scheduled step over all fronts of a tree level and all replicas.
//
// FP64: FP64 tensor-core MMA (mma.sync m8n8k4 .f64).  A complex product is
// written as one real product of twice the size: with A read as the real
// M x 2K matrix of interleaved (re, im) pairs and B expanded on the fly to the
// real 2K x 2N matrix whose 2x2 block for b = br + i bi is [[br, bi], [-bi, br]],
// the real result is exactly the interleaved complex C (4 real products per
// complex product, no Gauss trick, so the rounding is that of a plain FP64
// complex product).
//
// FP32: plain register-tiled SIMT kernel (the mixed-precision form).
#include "kernels.cuh"

namespace cl {
namespace {

constexpr int TM = kTileM;  // complex rows per CTA
constexpr int TN = kTileN;  // complex columns per CTA
constexpr int TK = 8;       // complex k per stage

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// 128 threads = 4 warps in a 2 x 2 layout; each warp owns 32 complex rows x
// 16 complex columns = 4 x 4 MMA tiles of 8 x 8 reals.
__global__ void __launch_bounds__(128) k_gemm_f64(const GemmDesc* __restrict__ ds, int d0, int d1,
                                                  double2* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const int di = find_desc(ds, d0, d1, blockIdx.x);
  const GemmDesc d = ds[di];
  const int t = blockIdx.x - d.blk0;
  const int row0 = (t / d.tilesN) * TM, col0 = (t % d.tilesN) * TN;
  double2* base = arena + blockIdx.y * stride;
  const double2* __restrict__ A = base + d.a;
  const double2* __restrict__ B = base + d.b;
  double2* C = base + d.c;

  __shared__ double2 As[TM][TK + 1];
  __shared__ double2 Bs[TK][TN + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 16;  // complex offsets inside the tile
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  for (int k0 = 0; k0 < d.K; k0 += TK) {
#pragma unroll
    for (int q = 0; q < (TM * TK) / 128; ++q) {
      const int idx = tid + 128 * q, r = idx / TK, kk = idx % TK;
      const int gr = row0 + r, gk = k0 + kk;
      As[r][kk] = (gr < d.M && gk < d.K) ? A[(int64_t)gr * d.lda + gk] : make_double2(0, 0);
    }
#pragma unroll
    for (int q = 0; q < (TK * TN) / 128; ++q) {
      const int idx = tid + 128 * q, kk = idx / TN, c = idx % TN;
      const int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (gk < d.K && gc < d.N) ? B[(int64_t)gk * d.ldb + gc] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK / 2; ++q) {
      const int kc = 2 * q + (tig >> 1);
      const bool imrow = tig & 1;  // real k index 2kc+1 (imaginary part of A)
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double2 a = As[wm + 8 * i + g][kc];
        af[i] = imrow ? a.y : a.x;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double2 b = Bs[kc][wn + 4 * j + (g >> 1)];
        const bool imcol = g & 1;  // real column 2n+1 (imaginary part of C)
        bf[j] = imrow ? (imcol ? b.x : -b.y) : (imcol ? b.y : b.x);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }

  const double sg = d.neg ? -1.0 : 1.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = row0 + wm + 8 * i + g, c = col0 + wn + 4 * j + tig;
      if (r >= d.M || c >= d.N) continue;
      if (d.rmask.hit(r) || d.cmask.hit(c)) continue;
      double2 v = make_double2(sg * acc[i][j][0], sg * acc[i][j][1]);
      double2* p = C + (int64_t)r * d.ldc + c;
      if (d.beta) v = cadd(v, *p);
      *p = v;
    }
}

// FP32 complex GEMM, 256 threads, each 4 rows x 2 columns of the 64 x 32 tile.
constexpr int TK32 = 16;
__global__ void __launch_bounds__(256) k_gemm_f32(const GemmDesc* __restrict__ ds, int d0, int d1,
                                                  float2* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const int di = find_desc(ds, d0, d1, blockIdx.x);
  const GemmDesc d = ds[di];
  const int t = blockIdx.x - d.blk0;
  const int row0 = (t / d.tilesN) * TM, col0 = (t % d.tilesN) * TN;
  float2* base = arena + blockIdx.y * stride;
  const float2* __restrict__ A = base + d.a;
  const float2* __restrict__ B = base + d.b;
  float2* C = base + d.c;
  __shared__ float2 As[TK32][TM + 1];
  __shared__ float2 Bs[TK32][TN + 1];
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;  // 16 x 16 threads: rows tr + 16 i, cols tc + 16 j
  float2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < d.K; k0 += TK32) {
#pragma unroll
    for (int q = 0; q < (TM * TK32) / 256; ++q) {
      const int idx = tid + 256 * q, r = idx / TK32, kk = idx % TK32;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < d.M && gk < d.K) ? A[(int64_t)gr * d.lda + gk] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < (TK32 * TN) / 256; ++q) {
      const int idx = tid + 256 * q, kk = idx / TN, c = idx % TN;
      const int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (gk < d.K && gc < d.N) ? B[(int64_t)gk * d.ldb + gc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK32; ++kk) {
      float2 a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const float sg = d.neg ? -1.f : 1.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = row0 + tr + 16 * i, c = col0 + tc + 16 * j;
      if (r >= d.M || c >= d.N) continue;
      if (d.rmask.hit(r) || d.cmask.hit(c)) continue;
      float2 v = make_float2(sg * acc[i][j].x, sg * acc[i][j].y);
      float2* p = C + (int64_t)r * d.ldc + c;
      if (d.beta) {
        v.x += p->x;
        v.y += p->y;
      }
      *p = v;
    }
}

}  // namespace

cudaError_t launch_gemm(const Plan& p, const Op& op, double2* arena, cudaStream_t st) {
  if (digit_gemms(p.precision)) return launch_gemm_emu(p, op, arena, st);
  const dim3 grid((unsigned)op.blocks, (unsigned)p.fbatch);
  return launch_k(k_gemm_f64, grid, dim3(128), 0, st, op_launch(p, op), p.d_gemm, op.d0, op.d1, arena,
                  p.arena_elems);
}

cudaError_t launch_gemm(const Plan& p, const Op& op, float2* arena, cudaStream_t st) {
  const dim3 grid((unsigned)op.blocks, (unsigned)p.fbatch);
  return launch_k(k_gemm_f32, grid, dim3(256), 0, st, op_launch(p, op), p.d_gemm, op.d0, op.d1, arena,
                  p.arena_elems);
}

}  // namespace cl
