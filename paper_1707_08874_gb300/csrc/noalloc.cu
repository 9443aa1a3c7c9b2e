// Allocation-free drift evaluation for small lattices.
//
// Some callers cannot allocate device memory at the point where they need a
// drift: host runtimes whose device memory is owned and budgeted by another
// allocator (a framework's caching allocator that has reserved the GPU), or
// plugins and embedded solvers that must not grow the process's footprint
// per call, or loops that cannot afford cudaMalloc / cudaFree, which may
// synchronise the whole device.  cl_drift_eval_noalloc serves them: all the
// scratch memory the factorisation and the selected inversion need (fronts,
// workspace, index tables, status word) lives in one file-scope device array
// of fixed size that every GPU loading this library holds until the process
// exits.  The paper has no counterpart; it is a deployment convenience.
//
// Set-up work: the first call on a device looks up the array's device
// address (cudaGetSymbolAddress), and the first call for a lattice shape on a
// device analyses the shape on the host and uploads its index tables into the
// array; later calls with the same shape on that device reuse both, so they
// issue only a status-word clear and the kernels.  Make those first calls
// before any stream capture.  The cached address belongs to the device's
// context: after cudaDeviceReset the entry point must not be called again in
// the same process.
#include <mutex>
#include <new>
#include <stdexcept>

#include "kernels.cuh"

namespace {

// Maximum scratch: 20 MiB.  A 4^4 lattice (V = 256) needs ~14.5 MiB; larger
// shapes are rejected with CL_ERR_UNSUPPORTED before any device work.
constexpr size_t kNoAllocBytes = 20u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// the shape whose tables are resident in a device's scratch array, and its
// host plan (op lists and descriptor tables)
struct Resident {
  int Ns = 0, Nt = 0;
  cl::Plan plan;
  size_t arena_bytes = 0;
};
Resident* g_resident[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device.  The symbol name
// is only a host-side handle; the address must be queried on each device.
// Called with g_mutex held.
int scratch_address(int dev, unsigned char** out) {
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return CL_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return CL_OK;
}

template <typename V>
cudaError_t place(unsigned char* base, size_t& off, V*& dst, const void* src, size_t bytes, cudaStream_t st) {
  dst = reinterpret_cast<V*>(base + off);
  off = align256(off + (bytes ? bytes : 16));
  if (!bytes) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}

// Analyses (Ns, Nt), checks that it fits the array and uploads its tables on
// `stream`, synchronising the stream so that the pageable host tables have
// reached the device before they go out of scope.  Called with g_mutex held.
int make_resident(int dev, int Ns, int Nt, unsigned char* base, cudaStream_t stream) {
  Resident* r = new (std::nothrow) Resident();
  if (!r) return CL_ERR_OOM;
  cl::Plan& p = r->plan;
  try {
    cl::analyze_host(p, Ns, Nt, 1, CL_FP64);
  } catch (const std::invalid_argument&) {
    delete r;
    return CL_ERR_INVALID_ARG;
  } catch (...) {
    delete r;
    return CL_ERR_UNSUPPORTED;
  }
  // layout inside the scratch array: status | arena | tables
  std::vector<int64_t> off;
  off.insert(off.end(), p.off_diag.begin(), p.off_diag.end());
  off.insert(off.end(), p.off_fwd.begin(), p.off_fwd.end());
  off.insert(off.end(), p.off_bwd.begin(), p.off_bwd.end());
  std::vector<int> ld;
  ld.insert(ld.end(), p.ld_diag.begin(), p.ld_diag.end());
  ld.insert(ld.end(), p.ld_fwd.begin(), p.ld_fwd.end());
  ld.insert(ld.end(), p.ld_bwd.begin(), p.ld_bwd.end());
  r->arena_bytes = align256((size_t)p.arena_elems * sizeof(double2));
  size_t need = 256 + r->arena_bytes;
  const size_t table_bytes[] = {off.size() * sizeof(int64_t), ld.size() * sizeof(int), p.maps.size() * sizeof(int),
                                p.gemm.size() * sizeof(cl::GemmDesc), p.panels.size() * sizeof(cl::PanelDesc),
                                p.copies.size() * sizeof(cl::CopyDesc), p.extadd.size() * sizeof(cl::ExtAddDesc),
                                p.gather.size() * sizeof(cl::GatherDesc), p.unperm.size() * sizeof(cl::UnpermDesc),
                                p.node_panels.size() * sizeof(int), (size_t)p.perm_ints * sizeof(int)};
  for (size_t b : table_bytes) need += align256(b ? b : 16);
  if (need > kNoAllocBytes) {
    delete r;
    return CL_ERR_UNSUPPORTED;
  }
  // the previous shape's tables are about to be overwritten
  delete g_resident[dev];
  g_resident[dev] = nullptr;
  p.d_status = reinterpret_cast<int*>(base);
  p.d_arena = base + 256;
  size_t o = 256 + r->arena_bytes;
  cudaError_t e = place(base, o, p.d_off, off.data(), table_bytes[0], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_ld, ld.data(), table_bytes[1], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_maps, p.maps.data(), table_bytes[2], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_gemm, p.gemm.data(), table_bytes[3], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_panels, p.panels.data(), table_bytes[4], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_copies, p.copies.data(), table_bytes[5], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_extadd, p.extadd.data(), table_bytes[6], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_gather, p.gather.data(), table_bytes[7], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_unperm, p.unperm.data(), table_bytes[8], stream);
  if (e == cudaSuccess) e = place(base, o, p.d_node_panels, p.node_panels.data(), table_bytes[9], stream);
  // the panels' row permutations (written by the panel kernels before they are read)
  p.d_perm = reinterpret_cast<int*>(base + o);
  o = align256(o + (table_bytes[10] ? table_bytes[10] : 16));
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    delete r;
    return CL_ERR_CUDA;
  }
  r->Ns = Ns;
  r->Nt = Nt;
  g_resident[dev] = r;
  return CL_OK;
}

}  // namespace

extern "C" int cl_drift_eval_noalloc(int Ns, int Nt, const double* links, double m, double mu, double nf,
                                     double* Gdiag, double* Gfwd, double* Gbwd, double* Kf,
                                     cudaStream_t stream) {
  if (!links || !Gfwd || !Gbwd || !Kf) return CL_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned char* base = nullptr;
  int st = scratch_address(dev, &base);
  if (st != CL_OK) return st;
  if (!g_resident[dev] || g_resident[dev]->Ns != Ns || g_resident[dev]->Nt != Nt) {
    if (cl::panel_prepare() != cudaSuccess) return CL_ERR_CUDA;
    st = make_resident(dev, Ns, Nt, base, stream);
    if (st != CL_OK) return st;
  }
  const cl::Plan& p = g_resident[dev]->plan;
  // the status word must start at zero; the fronts are cleared by the
  // schedule's first op
  cudaError_t e = cudaMemsetAsync(p.d_status, 0, 4 * sizeof(int), stream);
  if (e != cudaSuccess) return CL_ERR_CUDA;
  double2* arena = static_cast<double2*>(p.d_arena);
  for (const auto* ops : {&p.factor_ops, &p.selinv_ops})
    for (const auto& op : *ops) {
      if (op.blocks == 0 && op.kind != cl::OP_ZERO) continue;
      e = cl::launch_op<double2, double>(p, op, arena, links, m, mu, Gdiag, Gfwd, Gbwd, stream);
      if (e != cudaSuccess) return CL_ERR_CUDA;
    }
  e = cl::launch_drift(p, links, Gfwd, Gbwd, mu, nf, Kf, stream);
  return e == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}
