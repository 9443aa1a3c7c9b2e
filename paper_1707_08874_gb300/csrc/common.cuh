// Device helpers shared by the library's kernels: complex arithmetic on
// interleaved (re, im) pairs, lattice geometry and the CTA -> descriptor map.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"

namespace cl {

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

// Programmatic dependent launch.  Every kernel of the factorisation and the
// selected inversion starts here: it waits until the grids it depends on
// have completed and their writes are visible (a no-op for a kernel launched
// without the attribute), then lets its own successor in the stream start
// launching, so the successor's launch overlaps this kernel's run.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a += b * c
__device__ __forceinline__ void cfma(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, a.x);
  a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y);
  a.y = fma(b.y, c.x, a.y);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, a.x);
  a.x = fmaf(-b.y, c.y, a.x);
  a.y = fmaf(b.x, c.y, a.y);
  a.y = fmaf(b.y, c.x, a.y);
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
template <typename T> __device__ __forceinline__ T from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

// 3x3 complex matrices, row-major
struct M3 {
  double2 e[9];
};
__device__ __forceinline__ void load_m3(const double* p, M3& m) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = q[i];
}
__device__ __forceinline__ void store_m3(double* p, const M3& m) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int i = 0; i < 9; ++i) q[i] = m.e[i];
}
__device__ __forceinline__ M3 mul_m3(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(acc, a.e[3 * i + k], b.e[3 * k + j]);
      c.e[3 * i + j] = acc;
    }
  return c;
}
// inverse through the adjugate (cofactors) divided by the determinant
__device__ __forceinline__ M3 inv_m3(const M3& a) {
  const double2* A = a.e;
  M3 c;
  c.e[0] = csub(cmul(A[4], A[8]), cmul(A[5], A[7]));
  c.e[1] = csub(cmul(A[2], A[7]), cmul(A[1], A[8]));
  c.e[2] = csub(cmul(A[1], A[5]), cmul(A[2], A[4]));
  c.e[3] = csub(cmul(A[5], A[6]), cmul(A[3], A[8]));
  c.e[4] = csub(cmul(A[0], A[8]), cmul(A[2], A[6]));
  c.e[5] = csub(cmul(A[2], A[3]), cmul(A[0], A[5]));
  c.e[6] = csub(cmul(A[3], A[7]), cmul(A[4], A[6]));
  c.e[7] = csub(cmul(A[1], A[6]), cmul(A[0], A[7]));
  c.e[8] = csub(cmul(A[0], A[4]), cmul(A[1], A[3]));
  double2 det = cadd(cadd(cmul(A[0], c.e[0]), cmul(A[1], c.e[3])), cmul(A[2], c.e[6]));
  double n2 = det.x * det.x + det.y * det.y;
  double2 rdet = make_double2(det.x / n2, -det.y / n2);
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = cmul(c.e[i], rdet);
  return c;
}

struct LatticeGeo {
  int Ns, Nt, V;
  __device__ __forceinline__ void coords(int s, int c[4]) const {
    c[0] = s % Ns;
    s /= Ns;
    c[1] = s % Ns;
    s /= Ns;
    c[2] = s % Ns;
    c[3] = s / Ns;
  }
  // eta_nu(s) * s_nu(s): staggered phase times the antiperiodic temporal sign
  __device__ __forceinline__ double phase(int s, int nu) const {
    int c[4];
    coords(s, c);
    int sum = 0;
    for (int i = 0; i < nu; ++i) sum += c[i];
    double ph = (sum & 1) ? -1.0 : 1.0;
    if (nu == 3 && c[3] == Nt - 1) ph = -ph;
    return ph;
  }
};

// Last descriptor d in [d0, d1) with d.blk0 <= blk (descriptors sorted by blk0).
template <typename D>
__device__ __forceinline__ int find_desc(const D* __restrict__ ds, int d0, int d1, int blk) {
  int lo = d0, hi = d1 - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ds[mid].blk0 <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// status word: [0] code, [1] supernode, [2] column; [3] the largest pivot
// growth of the factorisation's panel blocks (float bits, see k_panel_inverse)
__device__ __forceinline__ void set_status(int* st, int code, int a, int b) {
  if (atomicCAS(st, 0, code) == 0) {
    st[1] = a;
    st[2] = b;
  }
}

}  // namespace cl
