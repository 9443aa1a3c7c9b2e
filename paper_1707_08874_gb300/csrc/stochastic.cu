// The stochastic estimator of the fermion drift (Eq. 7), the comparison path
// of the paper: tr[D^{-1} d_{axnu} D] ~ (1/n) sum_i eta_i^dag D^{-1} d_{axnu} D eta_i.
//
// With w_i = eta_i^dag D^{-1} (a row vector) the estimate of a link's drift is
// w_i[x] F_a eta_i[x+nu] + w_i[x+nu] B_a eta_i[x], i.e. the drift formula of
// Eq. 8 with the selected blocks replaced by their estimates
//   G_{x,x+nu} ~ (1/n) sum_i eta_i[x] w_i[x+nu]^T,  G_{x+nu,x} ~ (1/n) sum_i eta_i[x+nu] w_i[x]^T,
// whose expectation is exactly G for noise with E[eta eta^dag] = 1.
//
// The row vectors come from the factors that cl_factor leaves in the fronts:
// per front [[A_JJ^{-1}, U-hat], [-L-hat, Schur]] (U-hat = A_JJ^{-1} A_JS,
// L-hat = A_SJ A_JJ^{-1}).  Block elimination of w D = eta^dag gives
//   forward  (leaves to root): r_S <- r_S - r_J U-hat, passed to the parent
//            front (the extend-add of vectors);
//   backward (root to leaves): w_J = r_J A_JJ^{-1} + w_S (-L-hat), with w_S
//            read from the parent's front vector.
// Each front keeps its vector [J | S] of nf complex entries per noise vector
// in two workspaces (R forward, W backward); one launch per level and phase,
// one thread per output entry, deterministic (no atomics).
#include "kernels.cuh"

namespace cl {
namespace {

// node of a level launch that owns CTA `blk` (nodes of the level sorted by
// their first CTA)
template <bool kOverR>
__device__ __forceinline__ int find_vnode(const VecNode* __restrict__ vn, int v0, int v1, int blk) {
  int lo = v0, hi = v1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((kOverR ? vn[mid].blk_r : vn[mid].blk_nf) <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// forward, part 1: the front vectors of a level, R[e] = conj(eta) on the
// separator (e < k) plus the children's update vectors pulled through the
// extend-add site maps
__global__ void k_vec_assemble(const VecNode* __restrict__ vn, int v0, int v1, const int* __restrict__ maps,
                               const int* __restrict__ vsites, const double2* __restrict__ eta, int64_t sites,
                               int vrep, double2* __restrict__ R, int64_t vec_elems) {
  const int ni = find_vnode<false>(vn, v0, v1, blockIdx.x);
  const VecNode d = vn[ni];
  const int e = (blockIdx.x - d.blk_nf) * 128 + threadIdx.x;
  if (e >= d.nf) return;
  const int i = blockIdx.y, rep = blockIdx.z, n = gridDim.y;
  double2* Ri = R + ((int64_t)rep * n + i) * vec_elems;
  double2 v = make_double2(0, 0);
  if (e < d.k) {
    const int64_t site = (int64_t)rep * vrep + vsites[d.site0 + e / 3];
    v = cconj(eta[((int64_t)i * sites + site) * 3 + e % 3]);
  }
  for (int q = 0; q < d.nchild; ++q) {
    const int m = maps[d.ea_map[q] + e / 3];
    if (m >= 0) v = cadd(v, Ri[d.child_vec[q] + d.child_k[q] + 3 * m + e % 3]);
  }
  Ri[d.vec + e] = v;
}

// forward, part 2: the update vector r_S - r_J U-hat of every front of a
// level, in place over r_S (thread = entry s of S)
template <typename T>
__global__ void k_vec_update(const VecNode* __restrict__ vn, int v0, int v1, const T* __restrict__ arena,
                             int64_t stride, double2* __restrict__ R, int64_t vec_elems) {
  const int ni = find_vnode<true>(vn, v0, v1, blockIdx.x);
  const VecNode d = vn[ni];
  const int s = (blockIdx.x - d.blk_r) * 128 + threadIdx.x;
  if (s >= d.r) return;
  const int i = blockIdx.y, rep = blockIdx.z, n = gridDim.y;
  const double2* Ri = R + ((int64_t)rep * n + i) * vec_elems + d.vec;
  const T* F = arena + rep * stride + d.front + d.k + s;  // column k + s of the front
  double2 acc = Ri[d.k + s];
  double2 sub = make_double2(0, 0);
  for (int j = 0; j < d.k; ++j) cfma(sub, Ri[j], to_d2(F[(int64_t)j * d.nf]));
  R[((int64_t)rep * n + i) * vec_elems + d.vec + d.k + s] = csub(acc, sub);
}

// backward: W on the S part = the parent's W at the boundary sites; on the J
// part w_J = r_J A_JJ^{-1} + w_S (-L-hat), also written to the output w
template <typename T>
__global__ void k_vec_backward(const VecNode* __restrict__ vn, int v0, int v1, const int* __restrict__ maps,
                               const int* __restrict__ vsites, const T* __restrict__ arena, int64_t stride,
                               const double2* __restrict__ R, double2* __restrict__ W, int64_t vec_elems,
                               double2* __restrict__ w, int64_t sites, int vrep, const PanelDesc* __restrict__ pan,
                               const int* __restrict__ node_panels, const int* __restrict__ perm,
                               int64_t perm_stride) {
  const int ni = find_vnode<false>(vn, v0, v1, blockIdx.x);
  const VecNode d = vn[ni];
  const int e = (blockIdx.x - d.blk_nf) * 128 + threadIdx.x;
  if (e >= d.nf) return;
  const int i = blockIdx.y, rep = blockIdx.z, n = gridDim.y;
  const int64_t vb = ((int64_t)rep * n + i) * vec_elems;
  const double2* Ri = R + vb + d.vec;
  double2* Wi = W + vb;
  // w_S entry s: the parent's front vector at the position of boundary site s / 3
  auto wpar = [&](int s) { return Wi[d.parent_vec + 3 * maps[d.ga_map + s / 3] + s % 3]; };
  if (e >= d.k) {  // a boundary entry (a root has none)
    Wi[d.vec + e] = wpar(e - d.k);
    return;
  }
  const T* F = arena + rep * stride + d.front + e;  // column e of the front
  double2 acc = make_double2(0, 0);
  for (int j = 0; j < d.k; ++j) cfma(acc, Ri[j], to_d2(F[(int64_t)j * d.nf]));
  for (int s = 0; s < d.r; ++s) cfma(acc, wpar(s), to_d2(F[(int64_t)(d.k + s) * d.nf]));
  // the factors are those of the row-permuted supernode: entry e belongs to
  // its unknown pi(e), the panels' row exchanges composed (the last first)
  int x = e;
  const int* pm = perm + rep * perm_stride;
  for (int q = d.npan - 1; q >= 0; --q) {
    const PanelDesc pd = pan[node_panels[d.pan0 + q]];
    if (pd.nc > pd.bp && x >= pd.col0 && x < pd.col0 + pd.nc) x = pd.col0 + pm[pd.lperm + x - pd.col0];
  }
  Wi[d.vec + x] = acc;
  const int64_t site = (int64_t)rep * vrep + vsites[d.site0 + x / 3];
  w[((int64_t)i * sites + site) * 3 + x % 3] = acc;
}

// estimated selected blocks of one lattice shape: thread = link (s, nu)
__global__ void k_stoch_blocks(const double2* __restrict__ eta, const double2* __restrict__ w, int n, int64_t sites,
                               int64_t site_base, LatticeGeo g, double2* __restrict__ Gd, double2* __restrict__ Gf,
                               double2* __restrict__ Gb) {
  const int link = blockIdx.x * blockDim.x + threadIdx.x;
  if (link >= 4 * g.V) return;
  const int rep = blockIdx.y, s = link >> 2, nu = link & 3;
  int c[4];
  g.coords(s, c);
  c[nu] = (c[nu] + 1) % (nu == 3 ? g.Nt : g.Ns);
  const int y = ((c[3] * g.Ns + c[2]) * g.Ns + c[1]) * g.Ns + c[0];
  const int64_t xs = site_base + (int64_t)rep * g.V + s, ys = site_base + (int64_t)rep * g.V + y;
  double2 P[9], Q[9], Dg[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) P[q] = Q[q] = Dg[q] = make_double2(0, 0);
  for (int i = 0; i < n; ++i) {
    const double2* ei = eta + (int64_t)i * sites * 3;
    const double2* wi = w + (int64_t)i * sites * 3;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cfma(P[3 * a + b], ei[xs * 3 + a], wi[ys * 3 + b]);
        cfma(Q[3 * a + b], ei[ys * 3 + a], wi[xs * 3 + b]);
        if (nu == 0) cfma(Dg[3 * a + b], ei[xs * 3 + a], wi[xs * 3 + b]);
      }
  }
  const double inv = 1.0 / n;
  const int64_t o = ((int64_t)rep * g.V + s) * 4 + nu + site_base * 4;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    Gf[o * 9 + q] = cscale(P[q], inv);
    Gb[o * 9 + q] = cscale(Q[q], inv);
  }
  if (nu == 0 && Gd) {
    const int64_t od = site_base + (int64_t)rep * g.V + s;
#pragma unroll
    for (int q = 0; q < 9; ++q) Gd[od * 9 + q] = cscale(Dg[q], inv);
  }
}

}  // namespace

int64_t stochastic_work_elems(const Plan& p, int n) { return 2 * (int64_t)p.fbatch * n * p.vec_elems; }

// w = eta^dag D^{-1} for n noise vectors from the factors in the fronts
template <typename T>
cudaError_t launch_left_solve(const Plan& p, const double* eta, int n, double* w, double2* work, cudaStream_t st) {
  const T* arena = static_cast<const T*>(p.d_arena);
  const int64_t stride = p.arena_elems;
  const int64_t sites = p.ragged ? (int64_t)p.V : (int64_t)p.V * p.batch;
  const int vrep = p.ragged ? 0 : p.V;
  double2* R = work;
  double2* W = work + (int64_t)p.fbatch * n * p.vec_elems;
  const int nl = (int)p.vblk_nf.size();
  const double2* e2 = reinterpret_cast<const double2*>(eta);
  double2* w2 = reinterpret_cast<double2*>(w);
  for (int h = 0; h < nl; ++h) {  // forward, leaves to root
    const int v0 = p.vlevel[h], v1 = p.vlevel[h + 1];
    if (v1 == v0) continue;
    k_vec_assemble<<<dim3((unsigned)p.vblk_nf[h], (unsigned)n, (unsigned)p.fbatch), 128, 0, st>>>(
        p.d_vnodes, v0, v1, p.d_maps, p.d_vsites, e2, sites, vrep, R, p.vec_elems);
    if (p.vblk_r[h] > 0)
      k_vec_update<T><<<dim3((unsigned)p.vblk_r[h], (unsigned)n, (unsigned)p.fbatch), 128, 0, st>>>(
          p.d_vnodes, v0, v1, arena, stride, R, p.vec_elems);
  }
  for (int h = nl - 1; h >= 0; --h) {  // backward, root to leaves
    const int v0 = p.vlevel[h], v1 = p.vlevel[h + 1];
    if (v1 == v0) continue;
    k_vec_backward<T><<<dim3((unsigned)p.vblk_nf[h], (unsigned)n, (unsigned)p.fbatch), 128, 0, st>>>(
        p.d_vnodes, v0, v1, p.d_maps, p.d_vsites, arena, stride, R, W, p.vec_elems, w2, sites, vrep, p.d_panels,
        p.d_node_panels, p.d_perm, (int64_t)p.perm_ints);
  }
  return cudaGetLastError();
}
template cudaError_t launch_left_solve<double2>(const Plan&, const double*, int, double*, double2*, cudaStream_t);
template cudaError_t launch_left_solve<float2>(const Plan&, const double*, int, double*, double2*, cudaStream_t);

cudaError_t launch_stoch_blocks(const Plan& p, const double* eta, const double* w, int n, double* Gd, double* Gf,
                                double* Gb, cudaStream_t st) {
  const int64_t sites = p.ragged ? (int64_t)p.V : (int64_t)p.V * p.batch;
  for (const Segment& sg : p.segs) {
    const LatticeGeo g{sg.Ns, sg.Nt, sg.V};
    const dim3 grid((unsigned)((4 * sg.V + 127) / 128), (unsigned)sg.count);
    k_stoch_blocks<<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(eta), reinterpret_cast<const double2*>(w),
                                         n, sites, sg.site_base, g, reinterpret_cast<double2*>(Gd),
                                         reinterpret_cast<double2*>(Gf), reinterpret_cast<double2*>(Gb));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cl
