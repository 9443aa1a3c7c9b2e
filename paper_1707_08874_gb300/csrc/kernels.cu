// Element-wise and small dense kernels of the selected-inversion path:
// assembly of D into the fronts, extend-add, panel inverses, panel write-back,
// the gather of G_SS, extraction of the selected blocks and the fermion drift.
#include "kernels.cuh"

namespace cl {

// The per-link kernels take a block of kLinkBlock consecutive links and stage
// the block's 3x3 link-major records through shared memory: consecutive
// threads load (and store) consecutive 16-byte words, so every global access
// is coalesced; each thread then works on its own link's record.
constexpr int kLinkBlock = 128;
__device__ __forceinline__ void stage_in(const double2* __restrict__ src, int n, double2* __restrict__ sm) {
  for (int i = threadIdx.x; i < n; i += kLinkBlock) sm[i] = src[i];
}
__device__ __forceinline__ void stage_out(const double2* __restrict__ sm, int n, double2* __restrict__ dst) {
  for (int i = threadIdx.x; i < n; i += kLinkBlock) dst[i] = sm[i];
}

// ---------------------------------------------------------------------------
// D(m;mu) of Eq. 1 scattered into the fronts.  One thread per link (s, nu):
// D_{s,s+nu} = +1/2 eta s_nu e^{+mu} U,  D_{s+nu,s} = -1/2 eta s_nu e^{-mu} U^{-1}
// (e^{+-mu} on temporal hops only); the nu = 0 thread also writes D_{s,s} = m.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kLinkBlock) k_assemble(const double* __restrict__ links, T* __restrict__ arena,
                                                         int64_t stride, const int64_t* __restrict__ off,
                                                         const int* __restrict__ ld, LatticeGeo g, double m,
                                                         double mu, int* __restrict__ status) {
  pdl_enter();
  __shared__ double2 sm[kLinkBlock * 9];
  const int V = g.V, rep = blockIdx.y;
  const int l0 = blockIdx.x * kLinkBlock, nl = min(kLinkBlock, 4 * V - l0);
  stage_in(reinterpret_cast<const double2*>(links) + ((int64_t)rep * 4 * V + l0) * 9, nl * 9, sm);
  __syncthreads();
  const int link = l0 + threadIdx.x;
  if (threadIdx.x >= nl) return;
  const int s = link >> 2, nu = link & 3;
  T* A = arena + rep * stride;
  M3 u;
#pragma unroll
  for (int i = 0; i < 9; ++i) u.e[i] = sm[threadIdx.x * 9 + i];
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 9; ++i) finite = finite && isfinite(u.e[i].x) && isfinite(u.e[i].y);
  if (!finite) set_status(status, CL_ERR_NONFINITE, s, nu);  // a non-finite link (site, direction)
  M3 ui = inv_m3(u);
  const double ph = 0.5 * g.phase(s, nu);
  const double ef = nu == 3 ? exp(mu) : 1.0, eb = nu == 3 ? exp(-mu) : 1.0;
  const int64_t of = off[V + link], ob = off[5 * V + link];
  const int lf = ld[V + link], lb = ld[5 * V + link];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      A[of + a * lf + b] = from_d2<T>(cscale(u.e[3 * a + b], ph * ef));
      A[ob + a * lb + b] = from_d2<T>(cscale(ui.e[3 * a + b], -ph * eb));
    }
  if (nu == 0) {
    const int64_t od = off[s];
    const int l = ld[s];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) A[od + a * l + b] = from_d2<T>(make_double2(a == b ? m : 0.0, 0.0));
  }
}

// ---------------------------------------------------------------------------
// Extend-add, pull form: every parent front entry adds the Schur-complement
// entries of the children whose boundary contains both of its sites.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_extend_add(const ExtAddDesc* __restrict__ ds, int d0, int d1, const int* __restrict__ maps,
                             T* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const int di = find_desc(ds, d0, d1, blockIdx.x);
  const ExtAddDesc d = ds[di];
  const int64_t e = (int64_t)(blockIdx.x - d.blk0) * 256 + threadIdx.x;
  if (e >= (int64_t)d.nfp * d.nfp) return;
  const int i = (int)(e / d.nfp), j = (int)(e % d.nfp);
  T* A = arena + blockIdx.y * stride;
  double2 acc = make_double2(0, 0);
  bool any = false;
  for (int q = 0; q < d.nchild; ++q) {
    const int ci = maps[d.map[q] + i / 3], cj = maps[d.map[q] + j / 3];
    if (ci < 0 || cj < 0) continue;
    const int kc = d.kc[q];
    const T v = A[d.child[q] + (int64_t)(kc + 3 * ci + i % 3) * d.nfc[q] + kc + 3 * cj + j % 3];
    acc = cadd(acc, to_d2(v));
    any = true;
  }
  if (any) {
    T* p = A + d.parent + e;
    *p = from_d2<T>(cadd(to_d2(*p), acc));
  }
}

// ---------------------------------------------------------------------------
// Selected inversion, first step of a supernode: G_SS is read from the
// parent's front, which holds G on the parent's whole front after its own step.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather(const GatherDesc* __restrict__ ds, int d0, int d1, const int* __restrict__ maps,
                         T* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const int di = find_desc(ds, d0, d1, blockIdx.x);
  const GatherDesc d = ds[di];
  const int r = 3 * d.rs;
  const int64_t e = (int64_t)(blockIdx.x - d.blk0) * 256 + threadIdx.x;
  if (e >= (int64_t)r * r) return;
  const int i = (int)(e / r), j = (int)(e % r);
  T* A = arena + blockIdx.y * stride;
  const int pi = 3 * maps[d.map + i / 3] + i % 3, pj = 3 * maps[d.map + j / 3] + j % 3;
  A[d.child + (int64_t)(d.kc + i) * d.nfc + d.kc + j] = A[d.parent + (int64_t)pi * d.nfp + pj];
}

// ---------------------------------------------------------------------------
// Pivot panel of a supernode (bp <= kMaxPanel): its bp pivot rows are chosen
// among the rows of the panel and of the next panel of the supernode (partial
// pivoting on their panel columns), and the block of the chosen rows is
// inverted in place by Gauss-Jordan elimination with partial (row) pivoting
// inside it; those inner row interchanges are undone on the columns at the
// end, the exchange of rows between the two panels is kept (the row swap and
// the un-permutation after the selected inversion apply it).  Pivots are chosen by
// max(|re|, |im|), compared through the leading 32 bits of the ordered bit
// pattern of the absolute value (ties: the lowest row); a pivot below
// 1e-13 * max|block| (1e-6 for FP32 fronts) records CL_ERR_SINGULAR
// (supernode, column).
//
// A scalar FP64 warp instruction occupies a scheduler's FP64 unit for ~64
// cycles on this part (0.5 lanes per cycle, ~1.7 per SM), so every FP64 warp
// instruction should carry 32 live lanes and one code path: the update walks
// the bp x bp entries linearly with one FMA sequence per entry, and the
// kernel is instantiated per maximum panel width (24, 32, 48) so that its update
// loop holds only the slots that the width can fill.
// ---------------------------------------------------------------------------
constexpr int kMaxPanel = 48;

__device__ __forceinline__ long long mag_key(double2 v) {
  const long long a = __double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFll;
  const long long b = __double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFll;
  return a > b ? a : b;
}
__device__ __forceinline__ long long mag_key(float2 v) {
  const int a = __float_as_int(v.x) & 0x7FFFFFFF, b = __float_as_int(v.y) & 0x7FFFFFFF;
  return a > b ? a : b;
}
// 32-bit order key of the magnitude (monotone in max(|re|, |im|))
__device__ __forceinline__ unsigned key32(double2 v) { return (unsigned)(mag_key(v) >> 32); }
__device__ __forceinline__ unsigned key32(float2 v) { return (unsigned)mag_key(v); }
__device__ __forceinline__ double key_value(long long k, double) { return __longlong_as_double(k); }
__device__ __forceinline__ double key_value(long long k, float) { return (double)__int_as_float((int)k); }
__device__ __forceinline__ long long value_key(double v, double) { return __double_as_longlong(v); }
__device__ __forceinline__ long long value_key(double v, float) { return __float_as_int((float)v); }

// |x| truncated to single precision by integer operations (0 below the float
// range, +inf above): FP64 operations cost ~100 cycles of latency on this part
__device__ __forceinline__ float abs_to_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(b >> 52) - 1023 + 127;
  if (e <= 0) return 0.f;
  if (e >= 255) return __int_as_float(0x7F800000);
  return __int_as_float((e << 23) | (int)((b >> 29) & 0x7FFFFF));
}
// a finite, normal float as a double, by integer operations (exact)
__device__ __forceinline__ double float_to_double(float f) {
  const unsigned u = __float_as_uint(f);
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)(((u >> 23) & 0xFF) - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFF) << 29)));
}

// 1 / pv = conj(pv) / |pv|^2, branch-free.  FP64: a single-precision seed
// r0 of 1 / |pv|^2 formed from float copies of the components (integer
// conversions, beside the FP64 |pv|^2), e = 1 - |pv|^2 r0 (|e| < 2^-19) and
// conj(pv) r0 (1 + e + e^2), the series of 1 / (1 - e) cut below 2^-57:
// eight FP64 instructions in five dependent levels.  (Forming e as
// 1 - (x r0) x - (y r0) y saves one instruction and is more accurate per call,
// 1.7 against 3.0 ulp, but over twenty 4^4 lattices it left one at 1.4e-10
// of the G blocks, 2.7e-11 with this form, which keeps all twenty within
// 3.8e-11: kept out.)
// FP32: a fast reciprocal and one Newton step.  ok = false where
// the seed is unusable (zero, tiny, huge or non-finite pv); recip_exact then
// gives the plain quotient.
template <typename T, typename R>
__device__ __forceinline__ T recip_fast(T pv, bool& ok) {
  T inv;
  if (sizeof(R) == 8) {
    const float xf = abs_to_float(pv.x), yf = abs_to_float(pv.y);
    const float rf = __fdividef(1.0f, fmaf(xf, xf, yf * yf));
    ok = rf > 1e-30f && rf < 1e30f;  // normal, far from the float range limits
    const R r0 = ok ? (R)float_to_double(rf) : (R)0;
    const R n2 = fma(pv.x, pv.x, pv.y * pv.y);
    const R yx = pv.x * r0, yy = -pv.y * r0;
    const R e = fma(-n2, r0, (R)1);
    const R g = fma(e, e, e);
    inv.x = fma(yx, g, yx);
    inv.y = fma(yy, g, yy);
  } else {
    const R n2 = fma(pv.x, pv.x, pv.y * pv.y);
    ok = n2 > (R)1e-30 && n2 < (R)1e30;
    R r = __fdividef(1.0f, (float)n2);
    r = fma(r, fma(-n2, r, (R)1), r);
    inv.x = pv.x * r;
    inv.y = -pv.y * r;
  }
  return inv;
}
template <typename T, typename R>
__device__ __noinline__ T recip_exact(T pv) {
  const R r = (R)1 / fma(pv.x, pv.x, pv.y * pv.y);
  T inv;
  inv.x = pv.x * r;
  inv.y = -pv.y * r;
  return inv;
}

// pivot among logical rows c0..bp-1 of a column whose entry of logical row
// lane + 32 h the calling warp holds in v[h]: the largest magnitude key, the
// lowest row on ties
template <typename T, int H>
__device__ __forceinline__ int pivot_row(const T (&v)[H], int c0, int bp, int lane) {
  unsigned key = 0;
  int bi = 0x7fffffff;
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int i = lane + 32 * h;
    if (i < c0 || i >= bp) continue;
    const unsigned k = key32(v[h]);
    if (bi == 0x7fffffff || k > key) {
      key = k;
      bi = i;
    }
  }
  const unsigned kmax = __reduce_max_sync(0xffffffffu, bi != 0x7fffffff ? key : 0u);
  return (int)__reduce_min_sync(0xffffffffu, (bi != 0x7fffffff && key == kmax) ? (unsigned)bi : 0x7fffffffu);
}

// v - f w on complex entries, the one FMA sequence of every entry of a
// Gauss-Jordan step (the special rows and columns enter through their
// operands, not through a branch that would cost each warp both paths on the
// FP64 pipe)
template <typename T>
__device__ __forceinline__ T gj_fms(T v, T f, T w) {
  T r = v;
  r.x = fma(-f.x, w.x, r.x);
  r.x = fma(f.y, w.y, r.x);
  r.y = fma(-f.x, w.y, r.y);
  r.y = fma(-f.y, w.x, r.y);
  return r;
}

// logical rows a and b exchanged
__device__ __forceinline__ int swap_index(int i, int a, int b) { return i == a ? b : (i == b ? a : i); }

template <typename T>
constexpr size_t panel_smem_bytes(int mp) {
  // the block's two copies, then the candidate rows' panel columns (up to
  // 2 mp rows) in the front's precision and as float2 for the pivot choice
  return 2 * (size_t)mp * (mp + 1) * sizeof(T) + 2 * (size_t)mp * mp * sizeof(T) +
         2 * (size_t)mp * (mp + 1) * sizeof(float2);
}

__host__ __device__ constexpr int bit_count(unsigned m) { return m ? (int)(m & 1u) + bit_count(m >> 1) : 0; }

// Update-warp sets: warp w runs on scheduler w % 4.  The pivot chain of warp
// 0 is a string of dependent FP64 operations, and the SM's FP64 unit is one
// unit shared by its four schedulers (measured: ~1.7 lanes per cycle per SM,
// and one FP64 warp instruction per ~64 cycles per warp, whatever the number
// of live lanes); a chain instruction waits longer the more schedulers feed
// the unit (64 cycles alone, 95 with update warps on two schedulers, 133 on
// three).  So the update warps stay off scheduler 0, and 30-wide FP64 blocks
// keep them on two schedulers (one block: 55.3 us against 57.3 us on three).
constexpr unsigned kUpdNoSched0 = 0xEEEEu;
constexpr unsigned kUpdSched12 = 0x6666u;

// Gauss-Jordan step c in the scaled-multiplier form: with pivot p, column c
// values f_i and pivot row r_j (logical rows, before the step), every entry
// becomes v_ij - g_i w_j with g_i = f_i / p (g_c = -1/p), w_j = r_j (w_c = 1)
// and v = 0 on row c and column c, which yields the scaled pivot row r_j / p,
// the column -f_i / p and the pivot 1/p in one FMA sequence per entry.  The
// update warps read r_j from the step's input copy, so the chain only forms g.
//
// The block lives in two shared-memory copies: step c reads copy c & 1 and
// writes the other, so one barrier per column suffices.  Column look-ahead:
// while the update warps apply step c to every entry outside column c+1, warp
// 0 applies it to column c+1, every lane forms the reciprocal of its own
// candidate pivot while the pivot is chosen, and warp 0 leaves step c+1's row
// map and multipliers g for the next column (measured against the form that
// scales the pivot row on the chain: 24 / 30 / 48-wide FP64 blocks 36.9 / 55.3
// / 168 us against 41.0 / 59.1 / 212 us, FP32 14.3 / 16.4 / 38.9 against
// 17.4 / 22.4 / 53.3 us).  The row interchanges are undone at the end by
// reading the columns through the inverse of the final row map.
//
// CTAs np, np+1, ... of a launch run copy descriptors [x0, x1) instead (NT /
// 256 blocks of 256 entries each, xblocks in all): entries that the next
// products read and that no panel block of the launch holds.
template <typename T, typename R, int MP, int NT, unsigned UMASK>
__global__ void __launch_bounds__(NT)
    k_panel_inverse(const PanelDesc* __restrict__ ds, int d0, int np, const CopyDesc* __restrict__ cds, int x0, int x1,
                    int xblocks, T* __restrict__ arena, int64_t stride, int* __restrict__ perm, int64_t perm_stride,
                    int* __restrict__ status) {
  pdl_enter();
  if ((int)blockIdx.x >= np) {  // a copy CTA (CTA-uniform: no barrier on this path)
    const int cb = (NT / 256) * ((int)blockIdx.x - np) + (int)(threadIdx.x >> 8);
    if (cb >= xblocks) return;
    const CopyDesc x = cds[find_desc(cds, x0, x1, cb)];
    const int64_t e = (int64_t)(cb - x.blk0) * 256 + (threadIdx.x & 255);
    if (e >= (int64_t)x.rows * x.cols) return;
    const int i = (int)(e / x.cols), j = (int)(e % x.cols);
    if (x.rmask.hit(i) || x.cmask.hit(j)) return;
    T* B = arena + blockIdx.y * stride;
    B[x.dst + (int64_t)i * x.ldd + j] = B[x.src + (int64_t)i * x.lds + j];
    return;
  }
  constexpr int NU = bit_count(UMASK);                         // update warps
  constexpr int kSlots = (MP * MP + 32 * NU - 1) / (32 * NU);  // update entries per update thread
  constexpr int H = (MP + 31) / 32;                            // column entries per lane of warp 0
  constexpr int NW = NT / 32;
  static_assert((UMASK & 1u) == 0 && (UMASK >> NW) == 0, "update warps: 1 .. NT/32 - 1");
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T(*S)[MP][MP + 1] = reinterpret_cast<T(*)[MP][MP + 1]>(panel_smem);  // S[2]; logical row i in S[.][rmap[.][i]]
  __shared__ T gcol[2][MP];
  __shared__ int rmap[2][MP], qcol[MP];
  __shared__ long long wmax[NW], pkey[MP];
  T(*Tc)[MP] = reinterpret_cast<T(*)[MP]>(panel_smem + 2 * sizeof(T) * MP * (MP + 1));  // candidate rows
  float2(*Tf)[MP + 1] = reinterpret_cast<float2(*)[MP + 1]>(panel_smem + 2 * sizeof(T) * MP * (MP + 1) +
                                                            2 * sizeof(T) * MP * MP);  // rows padded: no bank conflicts
  __shared__ int lpl[2 * MP], chosen[MP], vlist[MP], ilist[MP];  // nc <= 2 MP candidate rows
  __shared__ unsigned char picked[2 * MP];
  __shared__ unsigned long long best[3];  // per column (mod 3): (magnitude bits << 32) | ~row
  // threads per candidate row in the pivot choice (a power of two, TPR 2 MP <= NT)
  constexpr int TPR = NT / (2 * MP) >= 8 ? 8 : (NT / (2 * MP) >= 4 ? 4 : (NT / (2 * MP) >= 2 ? 2 : 1));
  static_assert(TPR * 2 * MP <= NT, "one thread group per candidate row");
  const PanelDesc d = ds[d0 + blockIdx.x];
  T* A = arena + blockIdx.y * stride + d.a;
  const int bp = d.bp, nel = bp * bp, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nc = d.nc;  // candidate rows: this panel's and the next panel's
  const int srow = tid / TPR, ssub = tid % TPR;
  // Pivot rows.  Partial pivoting over the nc candidate rows of the panel's
  // columns chooses bp of them (in FP32: only the choice is taken from it);
  // the chosen rows of the panel keep their positions, the chosen rows of the
  // next panel take the positions of the panel rows left out, which move to
  // theirs (position i then holds candidate row lpl[i]).  The block inverted
  // below is that of the chosen rows.
  for (int e = tid; e < nc * bp; e += NT) {
    const int i = e / bp, j = e - i * bp;
    const T v = A[(int64_t)i * d.ld + j];
    Tc[i][j] = v;
    Tf[i][j] = make_float2((float)v.x, (float)v.y);
  }
  for (int i = tid; i < nc; i += NT) {
    lpl[i] = i;
    picked[i] = 0;
  }
  if (tid < 3) best[tid] = 0ull;
  __syncthreads();
  if (nc > bp) {
    // one barrier per column: each remaining row's group updates its row and
    // posts the row's magnitude in the next column through a shared atomic
    // maximum (ties: the lowest row), read after the barrier
    auto post = [&](int slot, int r, int col) {
      const float2 v = Tf[r][col];
      const unsigned m = max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y)));
      atomicMax(&best[slot], ((unsigned long long)m << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)r));
    };
    bool mine = srow < nc;  // this thread's row is still a candidate
    if (mine && ssub == 0) post(0, srow, 0);
    __syncthreads();
    for (int c = 0; c < bp; ++c) {
      const int pr = (int)(0xFFFFFFFFu - (unsigned)(best[c % 3] & 0xFFFFFFFFull));
      if (tid == 0) {
        chosen[c] = pr;
        best[(c + 2) % 3] = 0ull;  // read last at column c - 1, posted to from column c + 1 on
      }
      if (srow == pr) mine = false;
      if (mine && c + 1 < bp) {
        // eliminate column c from the row (fast reciprocal: only the choice is kept)
        const float2 pv = Tf[pr][c], v = Tf[srow][c];
        const float n2 = pv.x * pv.x + pv.y * pv.y;
        const float rn = n2 > 0.f ? __frcp_rn(n2) : 0.f;
        const float fr = (v.x * pv.x + v.y * pv.y) * rn, fi = (v.y * pv.x - v.x * pv.y) * rn;
        for (int j = c + 1 + ssub; j < bp; j += TPR) {
          const float2 w = Tf[pr][j];
          Tf[srow][j].x -= fr * w.x - fi * w.y;
          Tf[srow][j].y -= fr * w.y + fi * w.x;
        }
        if (ssub == 0) post((c + 1) % 3, srow, c + 1);  // its own update of column c + 1 is done
      }
      __syncthreads();
    }
    // pair the panel positions left out with the incoming rows (in pivot order)
    for (int c = tid; c < bp; c += NT) picked[chosen[c]] = 1;
    __syncthreads();
    if (warp == 0) {
      int nv = 0, ni = 0;
      for (int i0 = 0; i0 < bp; i0 += 32) {
        const int v = i0 + lane;
        const bool vac = v < bp && !picked[v];
        const bool inc = v < bp && chosen[v] >= bp;
        const unsigned mv = __ballot_sync(0xffffffffu, vac), mi = __ballot_sync(0xffffffffu, inc);
        const unsigned below = (1u << lane) - 1u;
        if (vac) vlist[nv + __popc(mv & below)] = v;
        if (inc) ilist[ni + __popc(mi & below)] = chosen[v];
        nv += __popc(mv);
        ni += __popc(mi);
      }
      __syncwarp();
      for (int q = lane; q < nv; q += 32) {  // nv == ni
        lpl[vlist[q]] = ilist[q];
        lpl[ilist[q]] = vlist[q];
      }
    }
    __syncthreads();
    int* lp = perm + blockIdx.y * perm_stride + d.lperm;
    for (int i = tid; i < nc; i += NT) lp[i] = lpl[i];
  }
  long long km = 0;
  for (int e = tid; e < nel; e += NT) {
    const int i = e / bp, j = e - i * bp;
    const T v = Tc[lpl[i]][j];
    S[0][i][j] = v;
    km = max(km, mag_key(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
  if (lane == 0) wmax[warp] = km;
  __syncthreads();
  // step 0's pivot, row map and multipliers
  if (warp == 0) {
    T v[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = lane + 32 * h;
      v[h] = i < bp ? S[0][i][0] : T{0, 0};
    }
    const int pr = pivot_row(v, 0, bp, lane);
    const T pv = S[0][pr][0];
    bool ok;
    T inv = recip_fast<T, R>(pv, ok);
    if (!ok) inv = recip_exact<T, R>(pv);  // pv is the same in every lane: warp-uniform
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = lane + 32 * h;
      if (i < bp) {
        const int s = swap_index(i, 0, pr);
        rmap[0][i] = s;
        gcol[0][i] = i == 0 ? T{-inv.x, -inv.y} : cmul(S[0][s][0], inv);
      }
    }
    if (lane == 0) pkey[0] = mag_key(pv);
  }
  // update entries: the thread of rank q among the update warps takes entries q, q + 32 NU, ...
  const bool upd = (UMASK >> warp) & 1u;
  const int rank = __popc(UMASK & ((1u << warp) - 1u));
  const int u = rank * 32 + lane;
  int ei[kSlots], ej[kSlots];
#pragma unroll
  for (int t = 0; t < kSlots; ++t) {
    const int e = u + 32 * NU * t;
    ei[t] = (upd && e < nel) ? e / bp : -1;
    ej[t] = ei[t] >= 0 ? e - ei[t] * bp : 0;
  }
  __syncthreads();
  for (int c = 0; c < bp; ++c) {
    const int cur = c & 1, nxt = cur ^ 1, cn = c + 1;
    const int rpc = rmap[cur][c];  // storage row of the pivot row
    if (warp == 0) {
      if (cn < bp) {
        // step c on column c+1 (logical row lane + 32 h in v[h])
        const T wc = S[cur][rpc][cn];
        T v[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int i = lane + 32 * h;
          v[h] = T{0, 0};
          if (i < bp) {
            const int r = rmap[cur][i];
            const T s0 = S[cur][r][cn];
            v[h] = gj_fms(i == c ? T{0, 0} : s0, gcol[cur][i], wc);
            S[nxt][r][cn] = v[h];
          }
        }
        // every lane's candidate reciprocal, beside the pivot search
        T rv[H];
        bool rok[H];
#pragma unroll
        for (int h = 0; h < H; ++h) rv[h] = recip_fast<T, R>(v[h], rok[h]);
        const int pr = pivot_row(v, cn, bp, lane);
        T mine = v[0], minv = rv[0];
        bool mok = rok[0];
#pragma unroll
        for (int h = 1; h < H; ++h)
          if ((pr >> 5) == h) mine = v[h], minv = rv[h], mok = rok[h];
        T pv, inv;
        pv.x = __shfl_sync(0xffffffffu, mine.x, pr & 31);
        pv.y = __shfl_sync(0xffffffffu, mine.y, pr & 31);
        inv.x = __shfl_sync(0xffffffffu, minv.x, pr & 31);
        inv.y = __shfl_sync(0xffffffffu, minv.y, pr & 31);
        if (!__shfl_sync(0xffffffffu, mok, pr & 31)) inv = recip_exact<T, R>(pv);  // warp-uniform, rare
        // step c+1: logical rows c+1 and pr exchanged; multipliers of column c+1
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int j = lane + 32 * h;
          if (j < bp) {
            rmap[nxt][j] = rmap[cur][swap_index(j, cn, pr)];
            gcol[nxt][swap_index(j, cn, pr)] = j == pr ? T{-inv.x, -inv.y} : cmul(v[h], inv);
          }
        }
        if (lane == 0) pkey[cn] = mag_key(pv);
      }
    } else if (upd) {
      // step c on every entry outside column c+1: all loads, the FMAs, the stores
      T vv[kSlots], ww[kSlots], ff[kSlots];
      int rp[kSlots];
#pragma unroll
      for (int t = 0; t < kSlots; ++t) {
        if (rank * 32 + 32 * NU * t >= nel) continue;  // warp-uniform: no live entry in this slot
        const int i = ei[t] >= 0 ? ei[t] : 0, j = ej[t];
        rp[t] = rmap[cur][i];
        const T s0 = S[cur][rp[t]][j];
        const T r0 = S[cur][rpc][j];
        vv[t] = (i == c || j == c) ? T{0, 0} : s0;
        ww[t] = j == c ? T{1, 0} : r0;
        ff[t] = gcol[cur][i];
      }
#pragma unroll
      for (int t = 0; t < kSlots; ++t) {
        if (rank * 32 + 32 * NU * t >= nel) continue;
        vv[t] = gj_fms(vv[t], ff[t], ww[t]);
      }
#pragma unroll
      for (int t = 0; t < kSlots; ++t)
        if (rank * 32 + 32 * NU * t < nel && ei[t] >= 0 && ej[t] != cn) S[nxt][rp[t]][ej[t]] = vv[t];
    }
    __syncthreads();
  }
  // result column j = column qcol[j] of the logical rows, qcol = inverse of
  // the final row map; pivots below 1e-13 max|block| (1e-6 for FP32) reported
  const int fin = bp & 1, fmap = (bp - 1) & 1;
  if (tid < bp) qcol[rmap[fmap][tid]] = tid;
  if (warp == 1) {
    long long m = wmax[0];
    for (int w = 1; w < NW; ++w) m = max(m, wmax[w]);
    const double rel = sizeof(R) == 8 ? 1e-13 : 1e-6;
    const long long thr = value_key(rel * key_value(m, R(0)), R(0));
    // a block holding an infinity or NaN (magnitude key at or above the
    // infinity's) is reported as non-finite, not as a tiny pivot
    const long long inf_key = sizeof(R) == 8 ? 0x7FF0000000000000ll : 0x7F800000ll;
    int bad = 0x7fffffff;
    long long pmin = 0x7FFFFFFFFFFFFFFFll;
    for (int c = lane; c < bp; c += 32) {
      if (pkey[c] < thr || pkey[c] == 0) bad = min(bad, c);
      pmin = min(pmin, pkey[c]);
    }
    bad = __reduce_min_sync(0xffffffffu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pmin = min(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
    if (lane == 0 && m >= inf_key) set_status(status, CL_ERR_NONFINITE, d.node, d.col0);
    else if (lane == 0 && bad != 0x7fffffff) set_status(status, CL_ERR_SINGULAR, d.node, d.col0 + bad);
    // pivot growth of the block: max |entry| / min |pivot| (magnitudes as
    // max(|re|, |im|)), kept as the largest over the factorisation in status[3]
    // (non-negative float bits order like the floats; a zero pivot gives +inf)
    if (lane == 0 && m < inf_key) {
      const double mv = key_value(m, R(0)), pv = key_value(pmin, R(0));
      const float ratio = pv > 0.0 ? (float)(mv / pv) : __int_as_float(0x7F800000);
      atomicMax(status + 3, __float_as_int(ratio));
    }
  }
  __syncthreads();
  for (int e = tid; e < nel; e += NT) {
    const int i = e / bp, j = e - i * bp;
    A[(int64_t)i * d.ld + j] = S[fin][rmap[fmap][i]][qcol[j]];
  }
  // the panel rows left out, now at the positions of the incoming rows (their
  // columns outside the panel are exchanged by the row swap after this launch)
  for (int e = bp * bp + tid; e < nc * bp; e += NT) {
    const int i = e / bp, j = e - i * bp;
    A[(int64_t)i * d.ld + j] = Tc[lpl[i]][j];
  }
}

// the instantiation for a plan's panel width (blocks of 24, 32 or 48): 512
// threads with the update warps off scheduler 0, on two schedulers for
// 32-wide FP64 blocks (measured per width and precision on one block)
template <typename T, typename R>
struct PanelLaunch {
  void (*k)(const PanelDesc*, int, int, const CopyDesc*, int, int, int, T*, int64_t, int*, int64_t, int*);
  int threads, block;
};
template <typename T, typename R>
PanelLaunch<T, R> panel_kernel(int panel) {
  if (panel <= 24) return {k_panel_inverse<T, R, 24, 512, kUpdNoSched0>, 512, 24};
  if (panel <= 32) {
    if constexpr (sizeof(R) == 8) return {k_panel_inverse<T, R, 32, 512, kUpdSched12>, 512, 32};
    return {k_panel_inverse<T, R, 32, 512, kUpdNoSched0>, 512, 32};
  }
  return {k_panel_inverse<T, R, kMaxPanel, 512, kUpdNoSched0>, 512, kMaxPanel};
}

// opt the panel kernels in to their dynamic shared memory on the current
// device (75 KB for 48-wide FP64 blocks; done before any launch or capture)
cudaError_t panel_prepare() {
  cudaError_t e = cudaSuccess;
  for (int w : {24, 32, kMaxPanel}) {
    const PanelLaunch<double2, double> pd = panel_kernel<double2, double>(w);
    const PanelLaunch<float2, float> pf = panel_kernel<float2, float>(w);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pd.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem_bytes<double2>(w));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pf.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem_bytes<float2>(w));
  }
  return e;
}

// ---------------------------------------------------------------------------
// Row exchanges of the cross-panel pivoting on the columns outside a panel.
// The panel's exchanges are disjoint pairs i <-> lperm[i] of its candidate
// rows.  A CTA takes kSwapCols columns of the front, and its kSwapGroups
// thread groups share out the pairs.  Each thread loads the entries of up to
// kSwapBatch pairs of its column before it stores any of them, so that those
// loads are in flight together.  Runs on the chain stream right after the
// panel inverse: the previous step's strips updated those rows on that stream,
// and its bulk update and write-back leave them out.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_swap_desc(const PanelDesc* __restrict__ ds, int d0, int d1, int blk) {
  int lo = d0, hi = d1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ds[mid].swap_blk0 <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
constexpr int kSwapGroups = 4;  // thread groups of a row-swap CTA, one pair in kSwapGroups each
constexpr int kSwapBatch = 8;   // pairs a thread loads before it stores them
template <typename T>
__global__ void __launch_bounds__(kSwapCols* kSwapGroups)
    k_row_swap(const PanelDesc* __restrict__ ds, int d0, int d1, const int* __restrict__ perm, int64_t perm_stride,
               T* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const PanelDesc d = ds[find_swap_desc(ds, d0, d1, blockIdx.x)];
  if (d.nc <= d.bp) return;  // CTA-uniform
  const int col = (blockIdx.x - d.swap_blk0) * kSwapCols + (int)(threadIdx.x % kSwapCols);
  const int grp = (int)(threadIdx.x / kSwapCols);
  // the panel's exchanged pairs (i < lperm[i]), listed once per CTA
  __shared__ int pair_i[2 * kMaxPanel], pair_j[2 * kMaxPanel], npairs;
  const int* lp = perm + blockIdx.y * perm_stride + d.lperm;
  if (threadIdx.x < 32) {
    int base = 0;
    for (int i0 = 0; i0 < d.nc; i0 += 32) {
      const int i = i0 + (int)threadIdx.x;
      const int j = i < d.nc ? lp[i] : -1;
      const bool take = j > i;
      const unsigned m = __ballot_sync(0xffffffffu, take);
      if (take) {
        const int q = base + __popc(m & ((1u << threadIdx.x) - 1u));
        pair_i[q] = i;
        pair_j[q] = j;
      }
      base += __popc(m);
    }
    if (threadIdx.x == 0) npairs = base;
  }
  __syncthreads();
  if (col >= d.ld || (col >= d.col0 && col < d.col0 + d.bp)) return;
  T* row0 = arena + blockIdx.y * stride + (d.a - d.col0) + col;  // column col of the first candidate row
  const int np = npairs;
  // the pairs are disjoint: no load of a batch reads an entry another pair stores
  for (int q0 = grp; q0 < np; q0 += kSwapGroups * kSwapBatch) {
    T a[kSwapBatch], b[kSwapBatch];
#pragma unroll
    for (int u = 0; u < kSwapBatch; ++u) {
      const int q = q0 + u * kSwapGroups;
      if (q < np) {
        a[u] = row0[(int64_t)pair_i[q] * d.ld];
        b[u] = row0[(int64_t)pair_j[q] * d.ld];
      } else {
        a[u] = b[u] = T{};
      }
    }
#pragma unroll
    for (int u = 0; u < kSwapBatch; ++u) {
      const int q = q0 + u * kSwapGroups;
      if (q < np) {
        row0[(int64_t)pair_i[q] * d.ld] = b[u];
        row0[(int64_t)pair_j[q] * d.ld] = a[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// After a supernode's selected-inversion step: its pivot-row columns back in
// the supernode's original order, by undoing its panels' row exchanges as
// column exchanges in reverse order (warp = front row).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(32 * kUnpermRows)
    k_unperm(const UnpermDesc* __restrict__ ds, int d0, int d1, const PanelDesc* __restrict__ pan,
             const int* __restrict__ node_panels, const int* __restrict__ perm, int64_t perm_stride,
             T* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const UnpermDesc d = ds[find_desc(ds, d0, d1, blockIdx.x)];
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x - d.blk0) * kUnpermRows + (threadIdx.x >> 5);
  if (row >= d.nf) return;
  T* F = arena + blockIdx.y * stride + d.front + (int64_t)row * d.nf;
  const int* pm = perm + blockIdx.y * perm_stride;
  for (int q = d.npan - 1; q >= 0; --q) {
    const PanelDesc pd = pan[node_panels[d.pan0 + q]];
    if (pd.nc <= pd.bp) continue;  // no exchange
    const int* lp = pm + pd.lperm;
    for (int i = lane; i < pd.nc; i += 32) {
      const int j = lp[i];
      if (j <= i) continue;
      const T a = F[pd.col0 + i], b = F[pd.col0 + j];
      F[pd.col0 + i] = b;
      F[pd.col0 + j] = a;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Strided block copy with row / column exclusion ranges.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_copy(const CopyDesc* __restrict__ ds, int d0, int d1, T* __restrict__ arena, int64_t stride) {
  pdl_enter();
  const int di = find_desc(ds, d0, d1, blockIdx.x);
  const CopyDesc d = ds[di];
  const int64_t e = (int64_t)(blockIdx.x - d.blk0) * 256 + threadIdx.x;
  if (e >= (int64_t)d.rows * d.cols) return;
  const int i = (int)(e / d.cols), j = (int)(e % d.cols);
  if (d.rmask.hit(i) || d.cmask.hit(j)) return;
  T* A = arena + blockIdx.y * stride;
  A[d.dst + (int64_t)i * d.ldd + j] = A[d.src + (int64_t)i * d.lds + j];
}

// ---------------------------------------------------------------------------
// Extraction of G_{s,s}, G_{s,s+nu}, G_{s+nu,s} from the fronts (same offsets
// as the assembly of the corresponding D blocks).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_extract(const T* __restrict__ arena, int64_t stride, const int64_t* __restrict__ off,
                          const int* __restrict__ ld, int V, double* __restrict__ Gdiag, double* __restrict__ Gfwd,
                          double* __restrict__ Gbwd) {
  pdl_enter();
  const int link = blockIdx.x * blockDim.x + threadIdx.x;
  if (link >= 4 * V) return;
  const int rep = blockIdx.y;
  const T* A = arena + rep * stride;
  const int64_t of = off[V + link], ob = off[5 * V + link];
  const int lf = ld[V + link], lb = ld[5 * V + link];
  const int64_t o = (int64_t)rep * 4 * V + link;
  double2* F = Gfwd ? reinterpret_cast<double2*>(Gfwd) + o * 9 : nullptr;
  double2* B = Gbwd ? reinterpret_cast<double2*>(Gbwd) + o * 9 : nullptr;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (F) F[3 * a + b] = to_d2(A[of + a * lf + b]);
      if (B) B[3 * a + b] = to_d2(A[ob + a * lb + b]);
    }
  if ((link & 3) == 0 && Gdiag) {
    const int s = link >> 2;
    const int64_t od = off[s];
    const int l = ld[s];
    double2* Dg = reinterpret_cast<double2*>(Gdiag) + ((int64_t)rep * V + s) * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Dg[3 * a + b] = to_d2(A[od + a * l + b]);
  }
}

// ---------------------------------------------------------------------------
// Fermion drift, Eq. 6 via Eq. 8.  With P = G_{s,s+nu}, Q = G_{s+nu,s} and
// d_a U = i lambda_a U, d_a U^{-1} = -i U^{-1} lambda_a:
//   Tr(P B_a) + Tr(Q F_a) = Tr(lambda_a M),
//   M = (i/2) eta s_nu [e^{-mu} P U^{-1} + e^{+mu} U Q],
// and Tr(lambda_a M) is read off the entries of M for the eight Gell-Mann
// matrices.  Non-finite drift records CL_ERR_NONFINITE.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLinkBlock) k_drift(const double* __restrict__ links,
                                                      const double* __restrict__ Gfwd,
                                                      const double* __restrict__ Gbwd, LatticeGeo g, double mu,
                                                      double nf, double* __restrict__ Kf,
                                                      int* __restrict__ status) {
  pdl_enter();
  __shared__ double2 sm[kLinkBlock * 9];
  const int l0 = blockIdx.x * kLinkBlock, nl = min(kLinkBlock, 4 * g.V - l0);
  const int64_t o0 = (int64_t)blockIdx.y * 4 * g.V + l0;  // first link of the block
  const int t = threadIdx.x, link = l0 + t;
  const bool live = t < nl;
  M3 u, P, Q;
  const double* src[3] = {links, Gfwd, Gbwd};
  M3* dst[3] = {&u, &P, &Q};
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // the block's U, G_{s,s+nu}, G_{s+nu,s} records in turn
    stage_in(reinterpret_cast<const double2*>(src[a]) + o0 * 9, nl * 9, sm);
    __syncthreads();
    if (live) {
#pragma unroll
      for (int i = 0; i < 9; ++i) dst[a]->e[i] = sm[t * 9 + i];
    }
    __syncthreads();
  }
  double2 K[8];
  bool finite = true;
  if (live) {
    const int s = link >> 2, nu = link & 3;
    const M3 ui = inv_m3(u);
    const M3 a = mul_m3(P, ui), b = mul_m3(u, Q);
    const double ef = nu == 3 ? exp(mu) : 1.0, eb = nu == 3 ? exp(-mu) : 1.0;
    const double ph = 0.5 * g.phase(s, nu) * nf;
    M3 M;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double2 v = cadd(cscale(a.e[i], eb), cscale(b.e[i], ef));
      M.e[i] = make_double2(-ph * v.y, ph * v.x);  // multiply by i * ph
    }
    const double2* m = M.e;
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    K[0] = cadd(m[3], m[1]);                                      // lambda_1
    K[1] = make_double2(-(m[1].y - m[3].y), m[1].x - m[3].x);      // lambda_2: i (M01 - M10)
    K[2] = csub(m[0], m[4]);                                      // lambda_3
    K[3] = cadd(m[6], m[2]);                                      // lambda_4
    K[4] = make_double2(-(m[2].y - m[6].y), m[2].x - m[6].x);      // lambda_5: i (M02 - M20)
    K[5] = cadd(m[7], m[5]);                                      // lambda_6
    K[6] = make_double2(-(m[5].y - m[7].y), m[5].x - m[7].x);      // lambda_7: i (M12 - M21)
    K[7] = cscale(csub(cadd(m[0], m[4]), cscale(m[8], 2.0)), r3);  // lambda_8
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sm[t * 8 + q] = K[q];
      finite = finite && isfinite(K[q].x) && isfinite(K[q].y);
    }
    if (!finite) set_status(status, CL_ERR_NONFINITE, s, nu);
  }
  __syncthreads();
  stage_out(sm, nl * 8, reinterpret_cast<double2*>(Kf) + o0 * 8);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T, typename R>
cudaError_t launch_op(const Plan& p, const Op& op, T* arena, const double* links, double m, double mu,
                      double* Gdiag, double* Gfwd, double* Gbwd, cudaStream_t st) {
  const int64_t stride = p.arena_elems;
  const dim3 grid1((unsigned)op.blocks, (unsigned)p.fbatch);
  const LaunchOpt prio = op_launch(p, op);
  switch (op.kind) {
    case OP_ZERO:
      return cudaMemset2DAsync(arena, (size_t)stride * sizeof(T), 0, (size_t)p.pool_elems * sizeof(T),
                               (size_t)p.fbatch, st);
    case OP_ASSEMBLE:
      // one launch per lattice shape: its replicas on grid.y, its links, fronts and block tables
      for (const Segment& sg : p.segs) {
        const LatticeGeo g{sg.Ns, sg.Nt, sg.V};
        const dim3 grid((unsigned)((4 * sg.V + kLinkBlock - 1) / kLinkBlock), (unsigned)sg.count);
        const cudaError_t e =
            launch_k(k_assemble<T>, grid, dim3(kLinkBlock), 0, st, prio, links + sg.site_base * 72, arena + sg.pool_base,
                     sg.rep_stride, p.d_off + sg.table_base, p.d_ld + sg.table_base, g, m, mu, p.d_status);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    case OP_EXTADD:
      return launch_k(k_extend_add<T>, grid1, dim3(256), 0, st, prio, p.d_extadd, op.d0, op.d1, p.d_maps, arena,
                      stride);
    case OP_PANEL: {
      // the panel inverses, then CTAs for the copies launched with them
      const PanelLaunch<T, R> pl = panel_kernel<T, R>(p.panel);
      const int per = pl.threads / 256;
      const dim3 grid((unsigned)(op.blocks + (op.xblocks + per - 1) / per), (unsigned)p.fbatch);
      return launch_k(pl.k, grid, dim3(pl.threads), panel_smem_bytes<T>(pl.block), st, prio, p.d_panels, op.d0,
                      op.blocks, p.d_copies, op.x0, op.x1, op.xblocks, arena, stride, p.d_perm,
                      (int64_t)p.perm_ints, p.d_status);
    }
    case OP_SWAP:
      return launch_k(k_row_swap<T>, grid1, dim3(kSwapCols * kSwapGroups), 0, st, prio, p.d_panels, op.d0, op.d1, p.d_perm,
                      (int64_t)p.perm_ints, arena, stride);
    case OP_UNPERM:
      return launch_k(k_unperm<T>, grid1, dim3(32 * kUnpermRows), 0, st, prio, p.d_unperm, op.d0, op.d1,
                      p.d_panels, p.d_node_panels, p.d_perm, (int64_t)p.perm_ints, arena, stride);
    case OP_GEMM:
      return launch_gemm(p, op, arena, st);
    case OP_COPY:
      return launch_k(k_copy<T>, grid1, dim3(256), 0, st, prio, p.d_copies, op.d0, op.d1, arena, stride);
    case OP_GATHER:
      k_gather<T><<<grid1, 256, 0, st>>>(p.d_gather, op.d0, op.d1, p.d_maps, arena, stride);
      break;
    case OP_EXTRACT:
      for (const Segment& sg : p.segs) {
        const dim3 grid((unsigned)((4 * sg.V + 127) / 128), (unsigned)sg.count);
        k_extract<T><<<grid, 128, 0, st>>>(arena + sg.pool_base, sg.rep_stride, p.d_off + sg.table_base,
                                           p.d_ld + sg.table_base, sg.V, Gdiag ? Gdiag + sg.site_base * 18 : nullptr,
                                           Gfwd ? Gfwd + sg.site_base * 72 : nullptr,
                                           Gbwd ? Gbwd + sg.site_base * 72 : nullptr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
  }
  return cudaGetLastError();
}

template cudaError_t launch_op<double2, double>(const Plan&, const Op&, double2*, const double*, double, double,
                                                double*, double*, double*, cudaStream_t);
template cudaError_t launch_op<float2, float>(const Plan&, const Op&, float2*, const double*, double, double,
                                              double*, double*, double*, cudaStream_t);

cudaError_t launch_drift(const Plan& p, const double* links, const double* Gfwd, const double* Gbwd, double mu,
                         double nf, double* Kf, cudaStream_t st) {
  for (const Segment& sg : p.segs) {
    const LatticeGeo g{sg.Ns, sg.Nt, sg.V};
    const dim3 grid((unsigned)((4 * sg.V + kLinkBlock - 1) / kLinkBlock), (unsigned)sg.count);
    const int64_t b = sg.site_base;
    k_drift<<<grid, kLinkBlock, 0, st>>>(links + b * 72, Gfwd + b * 72, Gbwd + b * 72, g, mu, nf, Kf + b * 64,
                                         p.d_status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cl
