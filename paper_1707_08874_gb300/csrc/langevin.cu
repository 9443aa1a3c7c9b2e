// Complex-Langevin step on the device (Sec. 2, Eq. 3-5; Sec. 4.1): gauge
// drift from the Wilson action, adaptive step, SL(3,C) link update with
// Gaussian noise, gauge cooling and the observables.  One thread per link or
// per site, all replicas in one launch (blockIdx.y = replica).
#include "kernels.cuh"

namespace cl {
namespace {

struct Geo4 {
  int Ns, Nt, V;
  __device__ __forceinline__ int shift(int s, int nu, int d) const {
    int c[4];
    int t = s;
    c[0] = t % Ns; t /= Ns;
    c[1] = t % Ns; t /= Ns;
    c[2] = t % Ns;
    c[3] = t / Ns;
    const int L = nu == 3 ? Nt : Ns;
    c[nu] = (c[nu] + d + L) % L;
    return ((c[3] * Ns + c[2]) * Ns + c[1]) * Ns + c[0];
  }
};

__device__ __forceinline__ M3 eye3() {
  M3 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = make_double2((i % 4 == 0) ? 1.0 : 0.0, 0.0);
  return r;
}
__device__ __forceinline__ M3 add3(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = cadd(a.e[i], b.e[i]);
  return r;
}
__device__ __forceinline__ M3 dagger3(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.e[3 * i + j] = make_double2(a.e[3 * j + i].x, -a.e[3 * j + i].y);
  return r;
}
__device__ __forceinline__ double2 tr3(const M3& a) { return cadd(cadd(a.e[0], a.e[4]), a.e[8]); }

// exp(X) by scaling and squaring of a degree-14 Taylor polynomial (Horner),
// after scaling the 1-norm below 1/4: truncation < 0.25^15/15! ~ 1e-21.
__device__ M3 exp3(const M3& X) {
  double nrm = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double c = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) c += hypot(X.e[3 * i + j].x, X.e[3 * i + j].y);
    nrm = fmax(nrm, c);
  }
  int s = 0;
  while (nrm > 0.25 && s < 60) {
    nrm *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  M3 Y;
#pragma unroll
  for (int i = 0; i < 9; ++i) Y.e[i] = cscale(X.e[i], sc);
  M3 R = eye3();
  for (int n = 14; n >= 1; --n) {  // R = I + Y R / n
    M3 T = mul_m3(Y, R);
#pragma unroll
    for (int i = 0; i < 9; ++i) T.e[i] = cscale(T.e[i], 1.0 / n);
    R = add3(eye3(), T);
  }
  for (int q = 0; q < s; ++q) R = mul_m3(R, R);
  return R;
}

// i sum_a c_a lambda_a for complex coefficients (standard Gell-Mann order)
__device__ M3 algebra3(const double2* c) {
  const double r3 = 0.57735026918962576451;
  M3 H;  // H = sum_a c_a lambda_a
  H.e[0] = cadd(c[2], cscale(c[7], r3));
  H.e[4] = cadd(cscale(c[2], -1.0), cscale(c[7], r3));
  H.e[8] = cscale(c[7], -2.0 * r3);
  // lambda_1, lambda_2 on (0,1)/(1,0): c1 - i c2 and c1 + i c2
  H.e[1] = make_double2(c[0].x + c[1].y, c[0].y - c[1].x);
  H.e[3] = make_double2(c[0].x - c[1].y, c[0].y + c[1].x);
  H.e[2] = make_double2(c[3].x + c[4].y, c[3].y - c[4].x);
  H.e[6] = make_double2(c[3].x - c[4].y, c[3].y + c[4].x);
  H.e[5] = make_double2(c[5].x + c[6].y, c[5].y - c[6].x);
  H.e[7] = make_double2(c[5].x - c[6].y, c[5].y + c[6].x);
  M3 X;
#pragma unroll
  for (int i = 0; i < 9; ++i) X.e[i] = make_double2(-H.e[i].y, H.e[i].x);  // times i
  return X;
}

// Tr(lambda_a M), a = 1..8
__device__ __forceinline__ void gm_traces(const M3& M, double2* K) {
  const double2* m = M.e;
  const double r3 = 0.57735026918962576451;
  K[0] = cadd(m[3], m[1]);
  K[1] = make_double2(-(m[1].y - m[3].y), m[1].x - m[3].x);
  K[2] = csub(m[0], m[4]);
  K[3] = cadd(m[6], m[2]);
  K[4] = make_double2(-(m[2].y - m[6].y), m[2].x - m[6].x);
  K[5] = cadd(m[7], m[5]);
  K[6] = make_double2(-(m[5].y - m[7].y), m[5].x - m[7].x);
  K[7] = cscale(csub(cadd(m[0], m[4]), cscale(m[8], 2.0)), r3);
}

// Philox4x32-10 (Salmon et al., SC'11)
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// max of non-negative doubles through their ordered bit patterns
__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double read_max(const unsigned long long* slot) {
  return __longlong_as_double((long long)*slot);
}

__device__ __forceinline__ M3 load_link(const double* base, int64_t rep, int V, int s, int nu) {
  M3 m;
  load_m3(base + ((rep * V + s) * 4 + nu) * 18, m);
  return m;
}

// ---------------------------------------------------------------------------
__global__ void k_invert_links(const double* __restrict__ U, double* __restrict__ Ui, int V) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const int64_t o = ((int64_t)blockIdx.y * 4 * V + l) * 18;
  M3 u;
  load_m3(U + o, u);
  store_m3(Ui + o, inv_m3(u));
}

// K^g = (i beta/6) sum_staples Tr[lambda_a (U A - A^{-1} U^{-1})]; accumulate
// into K when acc != 0 (K = K^f + K^g), else overwrite.
__global__ void k_gauge_drift(const double* __restrict__ U, const double* __restrict__ Ui, Geo4 g, double beta,
                              double* __restrict__ K, int acc) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * g.V) return;
  const int64_t rep = blockIdx.y;
  const int s = l >> 2, nu = l & 3;
  const int xn = g.shift(s, nu, +1);
  M3 S, T;
#pragma unroll
  for (int i = 0; i < 9; ++i) S.e[i] = T.e[i] = make_double2(0, 0);
  for (int mu = 0; mu < 4; ++mu) {
    if (mu == nu) continue;
    const int xm = g.shift(s, mu, +1), xd = g.shift(s, mu, -1), xnd = g.shift(xn, mu, -1);
    // upper staple A = U_{x+nu,mu} U^{-1}_{x+mu,nu} U^{-1}_{x,mu}; A^{-1} = U_{x,mu} U_{x+mu,nu} U^{-1}_{x+nu,mu}
    M3 A = mul_m3(mul_m3(load_link(U, rep, g.V, xn, mu), load_link(Ui, rep, g.V, xm, nu)),
                  load_link(Ui, rep, g.V, s, mu));
    M3 Ai = mul_m3(mul_m3(load_link(U, rep, g.V, s, mu), load_link(U, rep, g.V, xm, nu)),
                   load_link(Ui, rep, g.V, xn, mu));
    S = add3(S, A);
    T = add3(T, Ai);
    // lower staple B = U^{-1}_{x+nu-mu,mu} U^{-1}_{x-mu,nu} U_{x-mu,mu}; B^{-1} = U^{-1}_{x-mu,mu} U_{x-mu,nu} U_{x+nu-mu,mu}
    M3 B = mul_m3(mul_m3(load_link(Ui, rep, g.V, xnd, mu), load_link(Ui, rep, g.V, xd, nu)),
                  load_link(U, rep, g.V, xd, mu));
    M3 Bi = mul_m3(mul_m3(load_link(Ui, rep, g.V, xd, mu), load_link(U, rep, g.V, xd, nu)),
                   load_link(U, rep, g.V, xnd, mu));
    S = add3(S, B);
    T = add3(T, Bi);
  }
  const M3 u = load_link(U, rep, g.V, s, nu), ui = load_link(Ui, rep, g.V, s, nu);
  const M3 P = mul_m3(u, S), Q = mul_m3(T, ui);
  M3 M;
  const double f = beta / 6.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double2 v = csub(P.e[i], Q.e[i]);
    M.e[i] = make_double2(-f * v.y, f * v.x);  // (i beta/6) (U S - T U^{-1})
  }
  double2 k[8];
  gm_traces(M, k);
  double2* out = reinterpret_cast<double2*>(K) + (rep * 4 * g.V + l) * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) out[a] = acc ? cadd(out[a], k[a]) : k[a];
}

// K_max = max over links of (sum_a |K_a|^2)^{1/2}, per replica
__global__ void k_kmax(const double* __restrict__ K, int V, unsigned long long* __restrict__ slots,
                       int* __restrict__ status) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const double2* k = reinterpret_cast<const double2*>(K) + ((int64_t)blockIdx.y * 4 * V + l) * 8;
  double n2 = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) n2 += k[a].x * k[a].x + k[a].y * k[a].y;
  if (!isfinite(n2)) {
    set_status(status, CL_ERR_NONFINITE, -1, l);
    return;
  }
  atomic_max_pos(slots + 4 * blockIdx.y, sqrt(n2));
}

__device__ __forceinline__ double step_eps(double kmax, double eps_max, double kappa) {
  if (kappa <= 0 || !(kmax > 0)) return eps_max;
  return fmin(eps_max, kappa / kmax);
}

// U <- exp(i sum_a lambda_a (eps K_a + sqrt(eps) eta_a)) U, eta from Philox:
// counter (link, half, step, replica), key = seed; Box-Muller on u = (x + 1/2) 2^-32
__global__ void k_update(double* __restrict__ U, const double* __restrict__ K, int V, LangevinArgs a,
                         const unsigned long long* __restrict__ slots, const double* __restrict__ state) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * V) return;
  const int rep = blockIdx.y;
  const double eps = a.fixed_eps > 0 ? a.fixed_eps : step_eps(read_max(slots + 4 * rep), a.eps_max, a.kappa);
  const unsigned step = (unsigned)(a.fixed_eps > 0 ? a.step : (long long)state[4 * rep + 1]);
  const uint2 key = make_uint2((unsigned)(a.seed & 0xffffffffull), (unsigned)(a.seed >> 32));
  double eta[8];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint4 w = philox(make_uint4((unsigned)l, (unsigned)h, step, (unsigned)rep), key);
    const double u0 = ((double)w.x + 0.5) * 0x1p-32, u1 = ((double)w.y + 0.5) * 0x1p-32;
    const double u2 = ((double)w.z + 0.5) * 0x1p-32, u3 = ((double)w.w + 0.5) * 0x1p-32;
    const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    double s0, c0, s1, c1;
    sincospi(2.0 * u1, &s0, &c0);
    sincospi(2.0 * u3, &s1, &c1);
    const double sq2 = 1.41421356237309504880;
    eta[4 * h + 0] = sq2 * r0 * c0;
    eta[4 * h + 1] = sq2 * r0 * s0;
    eta[4 * h + 2] = sq2 * r1 * c1;
    eta[4 * h + 3] = sq2 * r1 * s1;
  }
  const double2* k = reinterpret_cast<const double2*>(K) + ((int64_t)rep * 4 * V + l) * 8;
  const double se = sqrt(eps);
  double2 c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) c[q] = make_double2(eps * k[q].x + se * eta[q], eps * k[q].y);
  const M3 R = exp3(algebra3(c));
  double2* up = reinterpret_cast<double2*>(U) + ((int64_t)rep * 4 * V + l) * 9;
  M3 u;
#pragma unroll
  for (int i = 0; i < 9; ++i) u.e[i] = up[i];
  M3 v = mul_m3(R, u);
  if (a.renorm_det) {
    // U <- U / det(U)^{1/3}, principal cube root |d|^{1/3} e^{i arg(d) / 3}
    const double2* E = v.e;
    const double2 d = cadd(cadd(cmul(E[0], csub(cmul(E[4], E[8]), cmul(E[5], E[7]))),
                                cmul(E[1], csub(cmul(E[5], E[6]), cmul(E[3], E[8])))),
                           cmul(E[2], csub(cmul(E[3], E[7]), cmul(E[4], E[6]))));
    const double rad = 1.0 / cbrt(hypot(d.x, d.y)), ang = -atan2(d.y, d.x) / 3.0;
    double sn, cs;
    sincos(ang, &sn, &cs);
    const double2 f = make_double2(rad * cs, rad * sn);
#pragma unroll
    for (int i = 0; i < 9; ++i) v.e[i] = cmul(v.e[i], f);
  }
  if (a.reunit) {
    // projection onto SU(3) (Sec. 4.2's reunitarisation): the first row
    // normalised, the second made orthogonal to it (Gram-Schmidt) and
    // normalised, the third the complex conjugate of their cross product
    double2* E = v.e;
    const double n0 = 1.0 / sqrt(E[0].x * E[0].x + E[0].y * E[0].y + E[1].x * E[1].x + E[1].y * E[1].y +
                                 E[2].x * E[2].x + E[2].y * E[2].y);
#pragma unroll
    for (int j = 0; j < 3; ++j) E[j] = cscale(E[j], n0);
    double2 c = make_double2(0, 0);  // u^dagger row1
#pragma unroll
    for (int j = 0; j < 3; ++j) c = cadd(c, cmul(make_double2(E[j].x, -E[j].y), E[3 + j]));
#pragma unroll
    for (int j = 0; j < 3; ++j) E[3 + j] = csub(E[3 + j], cmul(c, E[j]));
    const double n1 = 1.0 / sqrt(E[3].x * E[3].x + E[3].y * E[3].y + E[4].x * E[4].x + E[4].y * E[4].y +
                                 E[5].x * E[5].x + E[5].y * E[5].y);
#pragma unroll
    for (int j = 3; j < 6; ++j) E[j] = cscale(E[j], n1);
    const double2 w0 = csub(cmul(E[1], E[5]), cmul(E[2], E[4]));
    const double2 w1 = csub(cmul(E[2], E[3]), cmul(E[0], E[5]));
    const double2 w2 = csub(cmul(E[0], E[4]), cmul(E[1], E[3]));
    E[6] = make_double2(w0.x, -w0.y);
    E[7] = make_double2(w1.x, -w1.y);
    E[8] = make_double2(w2.x, -w2.y);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) up[i] = v.e[i];
}

// cooling gradient f_x = sum_nu [U_x U_x^dag - U_{x-nu}^dag U_{x-nu}] (traceless), per site
__global__ void k_cool_grad(const double* __restrict__ U, Geo4 g, double* __restrict__ F,
                            unsigned long long* __restrict__ slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int64_t rep = blockIdx.y;
  M3 f;
#pragma unroll
  for (int i = 0; i < 9; ++i) f.e[i] = make_double2(0, 0);
  for (int nu = 0; nu < 4; ++nu) {
    const M3 u = load_link(U, rep, g.V, s, nu);
    const M3 w = load_link(U, rep, g.V, g.shift(s, nu, -1), nu);
    const M3 a = mul_m3(u, dagger3(u)), b = mul_m3(dagger3(w), w);
#pragma unroll
    for (int i = 0; i < 9; ++i) f.e[i] = cadd(f.e[i], csub(a.e[i], b.e[i]));
  }
  const double2 t3 = cscale(tr3(f), 1.0 / 3.0);
  f.e[0] = csub(f.e[0], t3);
  f.e[4] = csub(f.e[4], t3);
  f.e[8] = csub(f.e[8], t3);
  double n2 = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) n2 += f.e[i].x * f.e[i].x + f.e[i].y * f.e[i].y;
  store_m3(F + (rep * g.V + s) * 18, f);
  atomic_max_pos(slots + 4 * rep + 1, sqrt(n2));
}

// Omega_x = exp(-alpha f_x), Omega_x^{-1} = exp(+alpha f_x), alpha = alpha0 / max|f|
__global__ void k_cool_omega(const double* __restrict__ F, int V, double alpha0,
                             const unsigned long long* __restrict__ slots, double* __restrict__ Om,
                             double* __restrict__ Omi) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const int64_t rep = blockIdx.y;
  const double fmax = read_max(slots + 4 * rep + 1);
  const double alpha = fmax > 0 ? alpha0 / fmax : 0.0;
  M3 f;
  load_m3(F + (rep * V + s) * 18, f);
  M3 X;
#pragma unroll
  for (int i = 0; i < 9; ++i) X.e[i] = cscale(f.e[i], -alpha);
  store_m3(Om + (rep * V + s) * 18, exp3(X));
#pragma unroll
  for (int i = 0; i < 9; ++i) X.e[i] = cscale(f.e[i], alpha);
  store_m3(Omi + (rep * V + s) * 18, exp3(X));
}

// U_{x,nu} <- Omega_x U_{x,nu} Omega_{x+nu}^{-1}
__global__ void k_cool_apply(double* __restrict__ U, Geo4 g, const double* __restrict__ Om,
                             const double* __restrict__ Omi, unsigned long long* __restrict__ slots) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 4 * g.V) return;
  const int64_t rep = blockIdx.y;
  const int s = l >> 2, nu = l & 3;
  M3 o, oi, u;
  load_m3(Om + (rep * g.V + s) * 18, o);
  load_m3(Omi + (rep * g.V + g.shift(s, nu, +1)) * 18, oi);
  u = load_link(U, rep, g.V, s, nu);
  store_m3(U + ((rep * g.V + s) * 4 + nu) * 18, mul_m3(mul_m3(o, u), oi));
}

__global__ void k_clear_slot(unsigned long long* slots, int which) {
  slots[4 * blockIdx.x + which] = 0ull;
}

// Observables, first pass: per-block partial sums (fixed order) of
// [plaq_s re,im | plaq_t re,im | poly re,im | poly_inv re,im | cond re,im | unitarity |
//  density re,im]; density = Tr(G_{x+t,x} dD_{x,x+t}/dmu + G_{x,x+t} dD_{x+t,x}/dmu)
constexpr int kObsBlock = 128;
constexpr int kObsN = 13;
__global__ void __launch_bounds__(kObsBlock) k_obs_partial(const double* __restrict__ U, const double* __restrict__ Ui,
                                                           const double* __restrict__ Gdiag,
                                                           const double* __restrict__ Gfwd,
                                                           const double* __restrict__ Gbwd, double chem, Geo4 g,
                                                           double* __restrict__ part) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rep = blockIdx.y;
  double v[kObsN];
#pragma unroll
  for (int q = 0; q < kObsN; ++q) v[q] = 0;
  if (s < g.V) {
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        // U_P = U_{x,mu} U_{x+mu,nu} U^{-1}_{x+nu,mu} U^{-1}_{x,nu}
        const M3 P = mul_m3(mul_m3(load_link(U, rep, g.V, s, mu), load_link(U, rep, g.V, g.shift(s, mu, 1), nu)),
                            mul_m3(load_link(Ui, rep, g.V, g.shift(s, nu, 1), mu), load_link(Ui, rep, g.V, s, nu)));
        const double2 t = tr3(P);
        const int o = nu == 3 ? 2 : 0;
        v[o] += t.x;
        v[o + 1] += t.y;
      }
    if (s < g.Ns * g.Ns * g.Ns) {  // Polyakov line from the t = 0 slice
      const int vs = g.Ns * g.Ns * g.Ns;
      M3 L = eye3(), Li = eye3();
      for (int t = 0; t < g.Nt; ++t) {
        L = mul_m3(L, load_link(U, rep, g.V, s + t * vs, 3));
        Li = mul_m3(load_link(Ui, rep, g.V, s + t * vs, 3), Li);
      }
      const double2 a = tr3(L), b = tr3(Li);
      v[4] = a.x;
      v[5] = a.y;
      v[6] = b.x;
      v[7] = b.y;
    }
    if (Gdiag) {
      M3 G;
      load_m3(Gdiag + (rep * g.V + s) * 18, G);
      const double2 t = tr3(G);
      v[8] = t.x;
      v[9] = t.y;
    }
    if (Gfwd && Gbwd) {
      // dD_{x,x+t}/dmu = D_{x,x+t} = 1/2 eta_t s_t e^{mu} U; dD_{x+t,x}/dmu = -D_{x+t,x} = 1/2 eta_t s_t e^{-mu} U^{-1}
      const LatticeGeo lg{g.Ns, g.Nt, g.V};
      const double ph = 0.5 * lg.phase(s, 3);
      M3 gf, gb;
      load_m3(Gfwd + ((rep * g.V + s) * 4 + 3) * 18, gf);
      load_m3(Gbwd + ((rep * g.V + s) * 4 + 3) * 18, gb);
      const double2 a = tr3(mul_m3(gb, load_link(U, rep, g.V, s, 3)));
      const double2 b = tr3(mul_m3(gf, load_link(Ui, rep, g.V, s, 3)));
      const double ef = ph * exp(chem), eb = ph * exp(-chem);
      v[11] = ef * a.x + eb * b.x;
      v[12] = ef * a.y + eb * b.y;
    }
    for (int nu = 0; nu < 4; ++nu) {
      const M3 u = load_link(U, rep, g.V, s, nu);
      double n2 = 0;
#pragma unroll
      for (int i = 0; i < 9; ++i) n2 += u.e[i].x * u.e[i].x + u.e[i].y * u.e[i].y;
      v[10] += n2 - 3.0;
    }
  }
  __shared__ double sh[kObsN][kObsBlock];
#pragma unroll
  for (int q = 0; q < kObsN; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kObsBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < kObsN; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kObsN) part[(rep * gridDim.x + blockIdx.x) * kObsN + threadIdx.x] = sh[threadIdx.x][0];
}

// Observables, second pass (one thread per replica, fixed order); optionally
// advances the Langevin state: t += eps, step += 1.
__global__ void k_obs_final(const double* __restrict__ part, int nblk, Geo4 g, double nf, int has_g,
                            const unsigned long long* __restrict__ slots, LangevinArgs a, double* __restrict__ state,
                            double* __restrict__ obs, int advance, int nrep) {
  const int rep = blockIdx.x * blockDim.x + threadIdx.x;
  if (rep >= nrep) return;
  double v[kObsN];
#pragma unroll
  for (int q = 0; q < kObsN; ++q) v[q] = 0;
  for (int b = 0; b < nblk; ++b)
#pragma unroll
    for (int q = 0; q < kObsN; ++q) v[q] += part[((int64_t)rep * nblk + b) * kObsN + q];
  const double V = g.V, vs = (double)g.Ns * g.Ns * g.Ns;
  double* o = obs + (int64_t)rep * kObsFields;
  o[0] = v[0] / (9.0 * V);  // (1/3) Tr U_P averaged over 3V spatial plaquettes
  o[1] = v[1] / (9.0 * V);
  o[2] = v[2] / (9.0 * V);
  o[3] = v[3] / (9.0 * V);
  o[4] = v[4] / (3.0 * vs);
  o[5] = v[5] / (3.0 * vs);
  o[6] = v[6] / (3.0 * vs);
  o[7] = v[7] / (3.0 * vs);
  o[8] = has_g ? nf * v[8] / V : 0.0;
  o[9] = has_g ? nf * v[9] / V : 0.0;
  o[10] = v[10] / (4.0 * V);
  const double kmax = read_max(slots + 4 * rep);
  o[11] = kmax;
  o[12] = o[13] = o[14] = o[15] = 0.0;
  o[16] = has_g ? nf * v[11] / V : 0.0;
  o[17] = has_g ? nf * v[12] / V : 0.0;
  o[18] = o[19] = 0.0;
  if (advance) {
    const double eps = a.fixed_eps > 0 ? a.fixed_eps : step_eps(kmax, a.eps_max, a.kappa);
    double* st = state + 4 * rep;
    st[0] += eps;
    st[1] += 1.0;
    st[2] = eps;
    o[12] = eps;
    o[13] = st[0];
    o[14] = st[1];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static dim3 grid_links(const Plan& p) { return dim3((unsigned)((4 * p.V + 127) / 128), (unsigned)p.batch); }
static dim3 grid_sites(const Plan& p) { return dim3((unsigned)((p.V + 127) / 128), (unsigned)p.batch); }

cudaError_t launch_gauge_drift(const Plan& p, const double* U, double* Ui, double beta, double* K, int acc,
                               cudaStream_t st) {
  const Geo4 g{p.Ns, p.Nt, p.V};
  k_invert_links<<<grid_links(p), 128, 0, st>>>(U, Ui, p.V);
  k_gauge_drift<<<grid_links(p), 128, 0, st>>>(U, Ui, g, beta, K, acc);
  return cudaGetLastError();
}

cudaError_t launch_kmax(const Plan& p, const double* K, unsigned long long* slots, cudaStream_t st) {
  k_clear_slot<<<p.batch, 1, 0, st>>>(slots, 0);
  k_kmax<<<grid_links(p), 128, 0, st>>>(K, p.V, slots, p.d_status);
  return cudaGetLastError();
}

cudaError_t launch_update(const Plan& p, double* U, const double* K, const LangevinArgs& a,
                          const unsigned long long* slots, const double* state, cudaStream_t st) {
  k_update<<<grid_links(p), 128, 0, st>>>(U, K, p.V, a, slots, state);
  return cudaGetLastError();
}

cudaError_t launch_cool(const Plan& p, double* U, int n_cool, double alpha0, double* F, double* Om, double* Omi,
                        unsigned long long* slots, cudaStream_t st) {
  const Geo4 g{p.Ns, p.Nt, p.V};
  for (int i = 0; i < n_cool; ++i) {
    k_clear_slot<<<p.batch, 1, 0, st>>>(slots, 1);
    k_cool_grad<<<grid_sites(p), 128, 0, st>>>(U, g, F, slots);
    k_cool_omega<<<grid_sites(p), 128, 0, st>>>(F, p.V, alpha0, slots, Om, Omi);
    k_cool_apply<<<grid_links(p), 128, 0, st>>>(U, g, Om, Omi, slots);
  }
  return cudaGetLastError();
}

cudaError_t launch_obs_partial(const Plan& p, const double* U, double* Ui, const double* Gdiag, const double* Gfwd,
                               const double* Gbwd, double mu, double* part, bool invert, cudaStream_t st) {
  const Geo4 g{p.Ns, p.Nt, p.V};
  if (invert) k_invert_links<<<grid_links(p), 128, 0, st>>>(U, Ui, p.V);
  const dim3 gs((unsigned)((p.V + kObsBlock - 1) / kObsBlock), (unsigned)p.batch);
  k_obs_partial<<<gs, kObsBlock, 0, st>>>(U, Ui, Gdiag, Gfwd, Gbwd, mu, g, part);
  return cudaGetLastError();
}

cudaError_t launch_obs_final(const Plan& p, const double* part, bool has_g, double nf, const unsigned long long* slots,
                             const LangevinArgs& a, double* state, double* obs, int advance, cudaStream_t st) {
  const Geo4 g{p.Ns, p.Nt, p.V};
  k_obs_final<<<(p.batch + 63) / 64, 64, 0, st>>>(part, (p.V + kObsBlock - 1) / kObsBlock, g, nf, has_g ? 1 : 0,
                                                  slots, a, state, obs, advance, p.batch);
  return cudaGetLastError();
}

int obs_partial_doubles(const Plan& p) { return ((p.V + kObsBlock - 1) / kObsBlock) * kObsN; }

}  // namespace cl
