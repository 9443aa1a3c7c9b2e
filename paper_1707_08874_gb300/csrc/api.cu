#include <algorithm>
#include <cstdint>
#include <cstdlib>
// C ABI of the library (declared in clselinv.h): plan creation, device memory
// of the plan, and the stream-ordered compute calls.
#include <cstring>
#include <new>
#include <stdexcept>

#include "kernels.cuh"

using cl::Plan;

struct cl_plan {
  Plan p;
};

namespace {

template <typename V>
cudaError_t upload(V*& dst, const void* src, size_t bytes, size_t& total) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)&dst, bytes);
  if (e != cudaSuccess) return e;
  total += bytes;
  return src ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaMemset(dst, 0, bytes);
}

void free_device(Plan& p) {
  if (!p.has_device) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p.device);
  cudaFree(p.d_arena);
  cudaFree(p.d_status);
  cudaFree(p.d_off);
  cudaFree(p.d_ld);
  cudaFree(p.d_maps);
  cudaFree(p.d_gemm);
  cudaFree(p.d_panels);
  cudaFree(p.d_unperm);
  cudaFree(p.d_node_panels);
  cudaFree(p.d_perm);
  cudaFree(p.d_copies);
  cudaFree(p.d_extadd);
  cudaFree(p.d_gather);
  cudaFree(p.d_emu);
  cudaFree(p.d_vnodes);
  cudaFree(p.d_vsites);
  cudaFree(p.d_emu_words);
  cudaFree(p.d_emu_ints);
  for (double* q : {p.d_Gdiag, p.d_Gfwd, p.d_Gbwd, p.d_K, p.d_Ui, p.d_F, p.d_Om, p.d_Omi, p.d_part}) cudaFree(q);
  cudaFree(p.d_slots);
  for (void* ev : p.op_events)
    if (ev) cudaEventDestroy((cudaEvent_t)ev);
  p.op_events.clear();
  for (void* ev : {p.fork_event, p.join_events[0], p.join_events[1]})
    if (ev) cudaEventDestroy((cudaEvent_t)ev);
  for (void* s : p.streams)
    if (s) cudaStreamDestroy((cudaStream_t)s);
  p.fork_event = p.join_events[0] = p.join_events[1] = nullptr;
  p.streams[0] = p.streams[1] = nullptr;
  cudaSetDevice(prev);
  p.has_device = false;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CL_OK;
  return e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA;
}

size_t elem_bytes(const Plan& p) { return p.precision == CL_MIXED_FP32 ? sizeof(float2) : sizeof(double2); }

int setup_device(Plan& p) {
  cudaGetDevice(&p.device);
  if (cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess) return CL_ERR_CUDA;
  if (const char* cs = std::getenv("CLSELINV_CHAIN_SMS"))  // SMs kept free of bulk GEMM CTAs (tuning)
    p.chain_sms = std::min(std::max(std::atoi(cs), 0), p.num_sms - 1);
  size_t total = 0;
  cudaError_t e;
  if ((e = cl::panel_prepare()) != cudaSuccess) return cuda_status(e);
  const size_t arena = (size_t)p.arena_elems * p.fbatch * elem_bytes(p);
  if ((e = cudaMalloc(&p.d_arena, arena)) != cudaSuccess) return cuda_status(e);
  total += arena;
  p.has_device = true;
  if ((e = upload(p.d_status, nullptr, 4 * sizeof(int), total)) != cudaSuccess ||
      (e = upload(p.d_off, p.off_all.data(), p.off_all.size() * sizeof(int64_t), total)) != cudaSuccess ||
      (e = upload(p.d_ld, p.ld_all.data(), p.ld_all.size() * sizeof(int), total)) != cudaSuccess ||
      (e = upload(p.d_maps, p.maps.data(), p.maps.size() * sizeof(int), total)) != cudaSuccess ||
      (e = upload(p.d_gemm, p.gemm.data(), p.gemm.size() * sizeof(cl::GemmDesc), total)) != cudaSuccess ||
      (e = upload(p.d_panels, p.panels.data(), p.panels.size() * sizeof(cl::PanelDesc), total)) != cudaSuccess ||
      (e = upload(p.d_unperm, p.unperm.data(), p.unperm.size() * sizeof(cl::UnpermDesc), total)) != cudaSuccess ||
      (e = upload(p.d_node_panels, p.node_panels.data(), p.node_panels.size() * sizeof(int), total)) !=
          cudaSuccess ||
      (e = upload(p.d_perm, nullptr, (size_t)p.perm_ints * p.fbatch * sizeof(int), total)) != cudaSuccess ||
      (e = upload(p.d_copies, p.copies.data(), p.copies.size() * sizeof(cl::CopyDesc), total)) != cudaSuccess ||
      (e = upload(p.d_extadd, p.extadd.data(), p.extadd.size() * sizeof(cl::ExtAddDesc), total)) != cudaSuccess ||
      (e = upload(p.d_gather, p.gather.data(), p.gather.size() * sizeof(cl::GatherDesc), total)) != cudaSuccess ||
      (e = upload(p.d_vnodes, p.vnodes.data(), p.vnodes.size() * sizeof(cl::VecNode), total)) != cudaSuccess ||
      (e = upload(p.d_vsites, p.vsites.data(), p.vsites.size() * sizeof(int), total)) != cudaSuccess)
    return cuda_status(e);
  // Langevin-step buffers (single-shape plans; a ragged plan evaluates drifts only)
  const size_t B = p.ragged ? 0 : p.batch, V = p.V;
  if ((e = upload(p.d_Gdiag, nullptr, B * V * 18 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_Gfwd, nullptr, B * V * 72 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_Gbwd, nullptr, B * V * 72 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_K, nullptr, B * V * 64 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_Ui, nullptr, B * V * 72 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_F, nullptr, B * V * 18 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_Om, nullptr, B * V * 18 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_Omi, nullptr, B * V * 18 * sizeof(double), total)) != cudaSuccess ||
      (e = upload(p.d_part, nullptr, B ? B * cl::obs_partial_doubles(p) * sizeof(double) : 0, total)) !=
          cudaSuccess ||
      (e = upload(p.d_slots, nullptr, B * 4 * sizeof(unsigned long long), total)) != cudaSuccess)
    return cuda_status(e);
  // streams and events of the two-stream factorisation
  bool two_streams = false;
  for (const auto& op : p.factor_ops) two_streams |= op.stream != 0;
  if (two_streams) {
    int lo = 0, hi = 0;
    cudaStream_t s0 = nullptr, s1 = nullptr;
    if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&s0, cudaStreamNonBlocking, hi)) != cudaSuccess)
      return cuda_status(e);
    p.streams[0] = s0;
    if ((e = cudaStreamCreateWithPriority(&s1, cudaStreamNonBlocking, lo)) != cudaSuccess) return cuda_status(e);
    p.streams[1] = s1;
    p.prio_lo = lo;
    p.prio_hi = hi;
    cudaEvent_t ev = nullptr;
    for (void** slot : {&p.fork_event, &p.join_events[0], &p.join_events[1]}) {
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
      *slot = ev;
    }
    p.op_events.assign(p.factor_ops.size(), nullptr);
    for (size_t i = 0; i < p.factor_ops.size(); ++i) {
      if (!p.factor_ops[i].signal) continue;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
      p.op_events[i] = ev;
    }
  }
  if (cl::digit_gemms(p.precision)) {
    if ((e = cl::emu_prepare()) != cudaSuccess) return cuda_status(e);
    if ((e = upload(p.d_emu, p.emu.data(), p.emu.size() * sizeof(cl::EmuDesc), total)) != cudaSuccess ||
        (e = upload(p.d_emu_words, nullptr, (size_t)p.fbatch * p.emu_words * sizeof(unsigned), total)) !=
            cudaSuccess ||
        (e = upload(p.d_emu_ints, nullptr, (size_t)p.fbatch * p.emu_ints * sizeof(int), total)) != cudaSuccess)
      return cuda_status(e);
  }
  p.device_bytes = total;
  return CL_OK;
}

bool compute_ready(const cl_plan* plan) { return plan && plan->p.has_device; }

const char* kFamilyName[cl::F_COUNT] = {"zero",  "assemble", "extend_add", "panel_inverse", "gemm",
                                         "copy",  "gather",   "extract",    "drift"};

// algorithmic work of one scheduled op over all replicas: flops of the complex
// products (8 real flops per complex multiply-add) and bytes that must cross
// DRAM (reads + writes of the data the op touches once)
void op_work(const Plan& p, const cl::Op& op, int& family, double& flops, double& bytes) {
  // B: replicas sharing each descriptor (grid.y); sites: of every lattice
  const double es = p.precision == CL_MIXED_FP32 ? 8.0 : 16.0, B = p.fbatch;
  const double sites = p.ragged ? p.V : (double)p.V * p.batch;
  flops = bytes = 0;
  switch (op.kind) {
    case cl::OP_ZERO: family = cl::F_ZERO; bytes = es * p.pool_elems * B; break;
    case cl::OP_ASSEMBLE: family = cl::F_ASSEMBLE; bytes = sites * (4 * 144.0 + (8 * 9 + 9) * es); break;
    case cl::OP_EXTADD:
      family = cl::F_EXTADD;
      for (int d = op.d0; d < op.d1; ++d) bytes += 3.0 * es * p.extadd[d].nfp * p.extadd[d].nfp * B;
      break;
    case cl::OP_PANEL:
      family = cl::F_PANEL;
      for (int d = op.d0; d < op.d1; ++d) {
        double bp = p.panels[d].bp;
        flops += 8.0 * bp * bp * bp * B;
        bytes += 2.0 * es * bp * bp * B;
      }
      for (int d = op.x0; d < op.x1; ++d) bytes += 2.0 * es * p.copies[d].rows * p.copies[d].cols * B;
      break;
    case cl::OP_GEMM:
      family = cl::F_GEMM;
      for (int d = op.d0; d < op.d1; ++d) {
        const cl::GemmDesc& g = p.gemm[d];
        flops += 8.0 * g.M * g.N * g.K * B;
        bytes += es * ((double)g.M * g.K + (double)g.K * g.N + (1.0 + g.beta) * g.M * g.N) * B;
      }
      break;
    case cl::OP_COPY:
      family = cl::F_COPY;
      for (int d = op.d0; d < op.d1; ++d) bytes += 2.0 * es * p.copies[d].rows * p.copies[d].cols * B;
      break;
    case cl::OP_GATHER:
      family = cl::F_GATHER;
      for (int d = op.d0; d < op.d1; ++d) bytes += 2.0 * es * 9.0 * p.gather[d].rs * p.gather[d].rs * B;
      break;
    case cl::OP_EXTRACT: family = cl::F_EXTRACT; bytes = sites * 9 * 9 * (es + 16.0); break;
    case cl::OP_SWAP:  // row exchanges of the cross-panel pivoting (counted with the copies)
      family = cl::F_COPY;
      for (int d = op.d0; d < op.d1; ++d)
        if (p.panels[d].nc > p.panels[d].bp) bytes += 2.0 * es * p.panels[d].nc * p.panels[d].ld * B;
      break;
    case cl::OP_UNPERM:
      family = cl::F_COPY;
      for (int d = op.d0; d < op.d1; ++d) bytes += 2.0 * es * p.unperm[d].nf * p.unperm[d].k * B;
      break;
  }
}

void prof_begin(Plan& p, cudaStream_t st, cudaEvent_t& e0) {
  e0 = nullptr;
  if (!p.profiling) return;
  cudaEventCreate(&e0);
  cudaEventRecord(e0, st);
}
void prof_end(Plan& p, cudaStream_t st, cudaEvent_t e0, int family, double flops, double bytes, int phase = -1,
              int idx = -1, int stream = 0, int level = -1) {
  if (!p.profiling || !e0) return;
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, st);
  p.prof.push_back(Plan::ProfRec{family, (void*)e0, (void*)e1, flops, bytes, phase, idx, stream, level});
}

template <typename T, typename R>
int launch_one(Plan& p, const cl::Op& op, T* arena, const double* links, double m, double mu, double* Gd,
               double* Gf, double* Gb, cudaStream_t st, int phase, int idx) {
  if (op.blocks == 0 && op.kind != cl::OP_ZERO) return CL_OK;
  cudaEvent_t e0;
  prof_begin(p, st, e0);
  cudaError_t e = cl::launch_op<T, R>(p, op, arena, links, m, mu, Gd, Gf, Gb, st);
  if (e != cudaSuccess) return cuda_status(e);
  if (p.profiling) {
    int fam;
    double fl, by;
    op_work(p, op, fam, fl, by);
    prof_end(p, st, e0, fam, fl, by, phase, idx, op.stream, op.level);
  }
  return CL_OK;
}

// Runs a schedule on the caller's stream.  A schedule with look-ahead (ops
// tagged for stream 1) runs on the plan's two streams: both are forked from
// the caller's stream, each op first waits for the op whose event it names,
// ops that signal record their event, and the caller's stream joins both at
// the end.  The same ops issued in list order on one stream give the same
// result (the list order is a valid sequential order).
template <typename T, typename R>
int run_ops(Plan& p, const std::vector<cl::Op>& ops, const double* links, double m, double mu, double* Gd,
            double* Gf, double* Gb, cudaStream_t st) {
  T* arena = static_cast<T*>(p.d_arena);
  const int phase = &ops == &p.factor_ops ? 0 : 1;
  const bool two = phase == 0 && p.streams[1] != nullptr;
  if (phase == 0) {  // the pivot growth word describes the latest factorisation
    const cudaError_t e0 = cudaMemsetAsync(p.d_status + 3, 0, sizeof(int), st);
    if (e0 != cudaSuccess) return cuda_status(e0);
  }
  // an op's first kernel may launch programmatically (overlapping its
  // predecessor's tail) only when it directly follows a kernel of this op list
  // on its stream, with no event wait in between
  // (never in a profiled run, whose per-kernel events would then overlap)
  auto launches_kernel = [](const cl::Op& op) { return op.kind != cl::OP_ZERO && op.blocks > 0; };
  if (!two) {
    bool fresh = true;
    for (size_t i = 0; i < ops.size(); ++i) {
      const cl::Op& op = ops[i];
      cl::Op o = op;
      o.pdl = !fresh && !p.profiling;
      const int r = launch_one<T, R>(p, o, arena, links, m, mu, Gd, Gf, Gb, st, phase, (int)i);
      if (r != CL_OK) return r;
      fresh = !launches_kernel(op);
    }
    return CL_OK;
  }
  cudaStream_t ss[2] = {(cudaStream_t)p.streams[0], (cudaStream_t)p.streams[1]};
  cudaError_t e = cudaEventRecord((cudaEvent_t)p.fork_event, st);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ss[k], (cudaEvent_t)p.fork_event, 0);
  if (e != cudaSuccess) return cuda_status(e);
  bool fresh[2] = {true, true};
  for (size_t i = 0; i < ops.size(); ++i) {
    const cl::Op& op = ops[i];
    cudaStream_t s = ss[op.stream];
    if (op.wait >= 0 && (e = cudaStreamWaitEvent(s, (cudaEvent_t)p.op_events[op.wait], 0)) != cudaSuccess)
      return cuda_status(e);
    cl::Op o = op;
    o.pdl = !fresh[op.stream] && op.wait < 0 && !p.profiling;
    fresh[op.stream] = !launches_kernel(op);
    const int r = launch_one<T, R>(p, o, arena, links, m, mu, Gd, Gf, Gb, s, phase, (int)i);
    if (r != CL_OK) return r;
    if (op.signal && (e = cudaEventRecord((cudaEvent_t)p.op_events[i], s)) != cudaSuccess) return cuda_status(e);
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventRecord((cudaEvent_t)p.join_events[k], ss[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, (cudaEvent_t)p.join_events[k], 0);
  }
  return cuda_status(e);
}

int run(Plan& p, const std::vector<cl::Op>& ops, const double* links, double m, double mu, double* Gd,
        double* Gf, double* Gb, cudaStream_t st) {
  if (p.precision == CL_MIXED_FP32) return run_ops<float2, float>(p, ops, links, m, mu, Gd, Gf, Gb, st);
  return run_ops<double2, double>(p, ops, links, m, mu, Gd, Gf, Gb, st);
}

int make_plan(int Ns, int Nt, int batch, int precision, int panel, cl_plan** out, bool device) {
  if (!out) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  if (device && batch < 1) return CL_ERR_INVALID_ARG;
  cl_plan* plan = new (std::nothrow) cl_plan();
  if (!plan) return CL_ERR_OOM;
  try {
    cl::analyze_host(plan->p, Ns, Nt, device ? batch : 1, precision, panel);
  } catch (const std::invalid_argument&) {
    delete plan;
    return CL_ERR_INVALID_ARG;
  } catch (const std::bad_alloc&) {
    delete plan;
    return CL_ERR_OOM;
  } catch (...) {
    delete plan;
    return CL_ERR_UNSUPPORTED;
  }
  if (device) {
    int st = setup_device(plan->p);
    if (st != CL_OK) {
      free_device(plan->p);
      delete plan;
      return st;
    }
  }
  *out = plan;
  return CL_OK;
}

int make_ragged(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, int panel,
                cl_plan** out, bool device = true) {
  if (!out) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  cl_plan* plan = new (std::nothrow) cl_plan();
  if (!plan) return CL_ERR_OOM;
  try {
    cl::analyze_ragged(plan->p, nshapes, Ns, Nt, count, precision, panel);
  } catch (const std::invalid_argument&) {
    delete plan;
    return CL_ERR_INVALID_ARG;
  } catch (const std::bad_alloc&) {
    delete plan;
    return CL_ERR_OOM;
  } catch (...) {
    delete plan;
    return CL_ERR_UNSUPPORTED;
  }
  int st = device ? setup_device(plan->p) : CL_OK;
  if (st != CL_OK) {
    free_device(plan->p);
    delete plan;
    return st;
  }
  *out = plan;
  return CL_OK;
}

// the Langevin pieces need one lattice shape (a ragged plan evaluates drifts)
bool langevin_ready(const cl_plan* plan) { return compute_ready(plan) && !plan->p.ragged; }

}  // namespace

extern "C" {

int cl_analyze_ragged(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, cl_plan** plan) {
  return make_ragged(nshapes, Ns, Nt, count, precision, 0, plan);
}

int cl_analyze_ragged_ex(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, int panel,
                         cl_plan** plan) {
  return make_ragged(nshapes, Ns, Nt, count, precision, panel, plan);
}

int cl_analyze_ragged_symbolic(int nshapes, const int* Ns, const int* Nt, const int* count, int precision, int panel,
                               cl_plan** plan) {
  return make_ragged(nshapes, Ns, Nt, count, precision, panel, plan, false);
}

int cl_analyze(int Ns, int Nt, int batch, int precision, cl_plan** plan) {
  return make_plan(Ns, Nt, batch, precision, 0, plan, true);
}

int cl_analyze_ex(int Ns, int Nt, int batch, int precision, int panel, cl_plan** plan) {
  return make_plan(Ns, Nt, batch, precision, panel, plan, true);
}

int cl_analyze_symbolic(int Ns, int Nt, int precision, cl_plan** plan) {
  return make_plan(Ns, Nt, 1, precision, 0, plan, false);
}

int cl_analyze_symbolic_ex(int Ns, int Nt, int precision, int panel, cl_plan** plan) {
  return make_plan(Ns, Nt, 1, precision, panel, plan, false);
}

int cl_factor(cl_plan* plan, const double* links, double m, double mu, cudaStream_t stream) {
  if (!compute_ready(plan) || !links) return CL_ERR_INVALID_ARG;
  return run(plan->p, plan->p.factor_ops, links, m, mu, nullptr, nullptr, nullptr, stream);
}

int cl_selinv_blocks(cl_plan* plan, double* Gdiag, double* Gfwd, double* Gbwd, cudaStream_t stream) {
  if (!compute_ready(plan)) return CL_ERR_INVALID_ARG;
  return run(plan->p, plan->p.selinv_ops, nullptr, 0, 0, Gdiag, Gfwd, Gbwd, stream);
}

int cl_fermion_drift(cl_plan* plan, const double* links, const double* Gfwd, const double* Gbwd, double mu,
                     double nf, double* Kf, cudaStream_t stream) {
  if (!compute_ready(plan) || !links || !Gfwd || !Gbwd || !Kf) return CL_ERR_INVALID_ARG;
  Plan& p = plan->p;
  cudaEvent_t e0;
  prof_begin(p, stream, e0);
  int st = cuda_status(cl::launch_drift(p, links, Gfwd, Gbwd, mu, nf, Kf, stream));
  const double sites = p.ragged ? p.V : (double)p.V * p.batch;
  prof_end(p, stream, e0, cl::F_DRIFT, 0.0, sites * 4 * (3 * 144.0 + 128.0));
  return st;
}

int cl_drift_eval(cl_plan* plan, const double* links, double m, double mu, double nf, double* Gdiag,
                  double* Gfwd, double* Gbwd, double* Kf, cudaStream_t stream) {
  if (!Gfwd || !Gbwd || !Kf) return CL_ERR_INVALID_ARG;
  int st = cl_factor(plan, links, m, mu, stream);
  if (st == CL_OK) st = cl_selinv_blocks(plan, Gdiag, Gfwd, Gbwd, stream);
  if (st == CL_OK) st = cl_fermion_drift(plan, links, Gfwd, Gbwd, mu, nf, Kf, stream);
  return st;
}

int cl_stochastic_workspace(const cl_plan* plan, int n, size_t* bytes) {
  if (!plan || n < 1 || !bytes) return CL_ERR_INVALID_ARG;
  *bytes = (size_t)cl::stochastic_work_elems(plan->p, n) * sizeof(double2);
  return CL_OK;
}

int cl_left_solve(cl_plan* plan, const double* eta, int n, double* w, void* work, size_t work_bytes,
                  cudaStream_t stream) {
  if (!compute_ready(plan) || !eta || !w || !work || n < 1 || n > 65535) return CL_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (work_bytes < (size_t)cl::stochastic_work_elems(p, n) * sizeof(double2) || ((uintptr_t)work & 15u))
    return CL_ERR_INVALID_ARG;
  double2* wk = static_cast<double2*>(work);
  const cudaError_t e = p.precision == CL_MIXED_FP32 ? cl::launch_left_solve<float2>(p, eta, n, w, wk, stream)
                                                     : cl::launch_left_solve<double2>(p, eta, n, w, wk, stream);
  return cuda_status(e);
}

int cl_stochastic_drift(cl_plan* plan, const double* links, double m, double mu, double nf, const double* eta, int n,
                        double* w, double* Gdiag_est, double* Gfwd_est, double* Gbwd_est, double* Kf, void* work,
                        size_t work_bytes, cudaStream_t stream) {
  if (!Gfwd_est || !Gbwd_est || !Kf) return CL_ERR_INVALID_ARG;
  int st = cl_factor(plan, links, m, mu, stream);
  if (st == CL_OK) st = cl_left_solve(plan, eta, n, w, work, work_bytes, stream);
  if (st == CL_OK)
    st = cuda_status(cl::launch_stoch_blocks(plan->p, eta, w, n, Gdiag_est, Gfwd_est, Gbwd_est, stream));
  if (st == CL_OK) st = cl_fermion_drift(plan, links, Gfwd_est, Gbwd_est, mu, nf, Kf, stream);
  return st;
}

int cl_gauge_drift(cl_plan* plan, const double* links, double beta, double* Kg, cudaStream_t stream) {
  if (!compute_ready(plan) || !links || !Kg) return CL_ERR_INVALID_ARG;
  if (!langevin_ready(plan)) return CL_ERR_UNSUPPORTED;
  return cuda_status(cl::launch_gauge_drift(plan->p, links, plan->p.d_Ui, beta, Kg, 0, stream));
}

int cl_gauge_cool(cl_plan* plan, double* links, int n_cool, double alpha0, cudaStream_t stream) {
  if (!compute_ready(plan) || !links || n_cool < 0) return CL_ERR_INVALID_ARG;
  if (!langevin_ready(plan)) return CL_ERR_UNSUPPORTED;
  Plan& p = plan->p;
  return cuda_status(cl::launch_cool(p, links, n_cool, alpha0, p.d_F, p.d_Om, p.d_Omi, p.d_slots, stream));
}

int cl_link_update(cl_plan* plan, double* links, const double* K, double eps, unsigned long long seed, long long step,
                   cudaStream_t stream) {
  if (!compute_ready(plan) || !links || !K || !(eps > 0)) return CL_ERR_INVALID_ARG;
  if (!langevin_ready(plan)) return CL_ERR_UNSUPPORTED;
  cl::LangevinArgs a{eps, 0.0, eps, seed, step};
  return cuda_status(cl::launch_update(plan->p, links, K, a, plan->p.d_slots, nullptr, stream));
}

int cl_observables(cl_plan* plan, const double* links, const double* Gdiag, const double* Gfwd, const double* Gbwd,
                   double mu, double nf, double* obs, cudaStream_t stream) {
  if (!compute_ready(plan) || !links || !obs) return CL_ERR_INVALID_ARG;
  if (!langevin_ready(plan)) return CL_ERR_UNSUPPORTED;
  Plan& p = plan->p;
  cl::LangevinArgs a{0.0, 0.0, 0.0, 0ull, 0};
  cudaError_t e = cl::launch_obs_partial(p, links, p.d_Ui, Gdiag, Gfwd, Gbwd, mu, p.d_part, true, stream);
  if (e == cudaSuccess)
    e = cl::launch_obs_final(p, p.d_part, Gdiag != nullptr, nf, p.d_slots, a, nullptr, obs, 0, stream);
  return cuda_status(e);
}

int cl_langevin_step(cl_plan* plan, double* links, const cl_langevin_params* prm, double* state, double* obs,
                     cudaStream_t stream) {
  if (!compute_ready(plan) || !links || !prm || !state || !obs) return CL_ERR_INVALID_ARG;
  if (!(prm->eps_max > 0) || prm->n_cool < 0) return CL_ERR_INVALID_ARG;
  if (!langevin_ready(plan)) return CL_ERR_UNSUPPORTED;
  Plan& p = plan->p;
  int st = CL_OK;
  const bool ferm = prm->fermions != 0;
  if (ferm) {
    st = cl_drift_eval(plan, links, prm->m, prm->mu, prm->nf, p.d_Gdiag, p.d_Gfwd, p.d_Gbwd, p.d_K, stream);
    if (st != CL_OK) return st;
  }
  cl::LangevinArgs a{prm->eps_max, prm->kappa, 0.0, prm->seed, 0};
  a.renorm_det = prm->renorm_det != 0;
  a.reunit = prm->reunit != 0;
  cudaError_t e = cl::launch_gauge_drift(p, links, p.d_Ui, prm->beta, p.d_K, ferm ? 1 : 0, stream);
  if (e == cudaSuccess) e = cl::launch_kmax(p, p.d_K, p.d_slots, stream);
  if (e == cudaSuccess)
    e = cl::launch_obs_partial(p, links, p.d_Ui, ferm ? p.d_Gdiag : nullptr, ferm ? p.d_Gfwd : nullptr,
                               ferm ? p.d_Gbwd : nullptr, prm->mu, p.d_part, false, stream);
  if (e == cudaSuccess) e = cl::launch_update(p, links, p.d_K, a, p.d_slots, state, stream);
  if (e == cudaSuccess && prm->n_cool > 0)
    e = cl::launch_cool(p, links, prm->n_cool, prm->alpha_cool, p.d_F, p.d_Om, p.d_Omi, p.d_slots, stream);
  if (e == cudaSuccess) e = cl::launch_obs_final(p, p.d_part, ferm, prm->nf, p.d_slots, a, state, obs, 1, stream);
  return cuda_status(e);
}

int cl_plan_set_wait_limit(cl_plan* plan, double seconds) {
  if (!plan) return CL_ERR_INVALID_ARG;
  if (seconds < 0) {
    plan->p.wait_ns = cl::kDefaultWaitNs;
  } else {
    const double ns = seconds * 1e9;
    plan->p.wait_ns = ns >= (double)cl::kDefaultWaitNs ? cl::kDefaultWaitNs : (unsigned long long)ns;
  }
  return CL_OK;
}

int cl_get_status(cl_plan* plan, cudaStream_t stream, int* info, int* detail) {
  if (!compute_ready(plan) || !info) return CL_ERR_INVALID_ARG;
  int h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h, plan->p.d_status, sizeof(h), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->p.d_status, 0, 3 * sizeof(int), stream);  // not the growth word
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e);
  *info = h[0];
  if (detail) {
    detail[0] = h[0] ? h[1] : -1;
    detail[1] = h[0] ? h[2] : -1;
  }
  return CL_OK;
}

int cl_plan_pivot_growth(cl_plan* plan, cudaStream_t stream, double* growth) {
  if (!compute_ready(plan) || !growth) return CL_ERR_INVALID_ARG;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, plan->p.d_status + 3, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e);
  float f;
  std::memcpy(&f, &h, sizeof(f));
  *growth = (double)f;
  return CL_OK;
}

int cl_plan_get_info(const cl_plan* plan, cl_plan_info* info) {
  if (!plan || !info) return CL_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  std::memset(info, 0, sizeof(*info));
  info->Ns = p.Ns;
  info->Nt = p.Nt;
  info->V = p.V;
  info->N = p.N;
  info->batch = p.batch;
  info->precision = p.precision;
  info->n_supernodes = (int)p.nodes.size();
  info->n_levels = p.n_levels;
  for (const auto& n : p.nodes) {
    info->max_front = std::max(info->max_front, n.nf);
    info->max_pivot_block = std::max(info->max_pivot_block, n.k);
  }
  info->panel = p.panel;
  info->factor_flops = p.factor_flops;
  info->selinv_flops = p.selinv_flops;
  info->front_bytes = (double)p.pool_elems * p.fbatch * elem_bytes(p);
  info->device_bytes = (double)p.device_bytes;
  const int nseg = (int)p.segs.size();
  int launches = nseg;  // drift, per lattice shape
  for (const auto* ops : {&p.factor_ops, &p.selinv_ops})
    for (const auto& op : *ops) {
      if (op.kind == cl::OP_ZERO || op.blocks == 0) continue;
      if (op.kind == cl::OP_ASSEMBLE || op.kind == cl::OP_EXTRACT) launches += nseg;
      else launches += (op.kind == cl::OP_GEMM && cl::digit_gemms(p.precision)) ? 2 : 1;  // split + GEMM
    }
  info->launches_per_eval = launches;
  info->workspace_bytes = (double)p.fbatch * (4.0 * p.emu_words + 4.0 * p.emu_ints);
  info->n_shapes = nseg;
  return CL_OK;
}

int cl_plan_check_schedule(const cl_plan* plan, int ignore_waits, long long* conflicts, char* first, int first_len) {
  if (!plan || !conflicts) return CL_ERR_INVALID_ARG;
  std::string msg;
  try {
    *conflicts = cl::check_factor_schedule(plan->p, ignore_waits != 0, &msg);
  } catch (const std::bad_alloc&) {
    return CL_ERR_OOM;
  }
  if (first && first_len > 0) {
    std::strncpy(first, msg.c_str(), (size_t)first_len - 1);
    first[first_len - 1] = 0;
  }
  return CL_OK;
}

int cl_plan_export(const cl_plan* plan, int table, long long* out, long long cap, long long* count) {
  if (!plan || !count || table < 0 || table > CL_TABLE_NODE_PANELS) return CL_ERR_INVALID_ARG;
  const cl::Plan& p = plan->p;
  std::vector<long long> v;
  auto mask = [&v](const cl::Mask2& m) { v.insert(v.end(), {m.r0, m.r1, m.r2, m.r3}); };
  switch (table) {
    case CL_TABLE_META:
      v = {p.Ns, p.Nt, p.V, p.N, p.precision, p.panel, p.pool_elems, p.tmp_elems, p.arena_elems, p.n_levels,
           p.perm_ints};
      break;
    case CL_TABLE_FACTOR_OPS:
    case CL_TABLE_SELINV_OPS:
      for (const auto& op : table == CL_TABLE_FACTOR_OPS ? p.factor_ops : p.selinv_ops)
        v.insert(v.end(),
                 {(long long)op.kind, op.d0, op.d1, op.blocks, op.level, op.stream, op.wait, op.signal, op.ndig,
                  op.x0, op.x1});
      break;
    case CL_TABLE_SEGMENTS:
      for (const auto& g : p.segs)
        v.insert(v.end(), {g.Ns, g.Nt, g.V, g.count, g.pool_base, g.rep_stride, g.table_base, g.site_base});
      break;
    case CL_TABLE_VNODES:
      for (const auto& x : p.vnodes)
        v.insert(v.end(), {x.front, x.vec, x.parent_vec, x.nf, x.k, x.r, x.level, x.nchild, x.child_vec[0],
                           x.child_vec[1], x.child_k[0], x.child_k[1], x.ea_map[0], x.ea_map[1], x.ga_map, x.site0,
                           x.pan0, x.npan});
      break;
    case CL_TABLE_VSITES:
      v.assign(p.vsites.begin(), p.vsites.end());
      break;
    case CL_TABLE_GEMM:
      for (const auto& g : p.gemm) {
        v.insert(v.end(), {g.a, g.b, g.c, g.lda, g.ldb, g.ldc, g.M, g.N, g.K, g.neg, g.beta});
        mask(g.rmask);
        mask(g.cmask);
        v.push_back(g.trans);
      }
      break;
    case CL_TABLE_PANEL:
      for (const auto& d : p.panels)
        v.insert(v.end(), {d.a, d.ld, d.bp, d.node, d.col0, d.nc, d.lperm, d.pi, d.swap_blk0});
      break;
    case CL_TABLE_UNPERM:
      for (const auto& d : p.unperm) v.insert(v.end(), {d.front, d.nf, d.k, d.pan0, d.npan, d.blk0});
      break;
    case CL_TABLE_NODE_PANELS:
      v.assign(p.node_panels.begin(), p.node_panels.end());
      break;
    case CL_TABLE_COPY:
      for (const auto& d : p.copies) {
        v.insert(v.end(), {d.src, d.dst, d.lds, d.ldd, d.rows, d.cols});
        mask(d.rmask);
        mask(d.cmask);
      }
      break;
    case CL_TABLE_EXTADD:
      for (const auto& d : p.extadd)
        v.insert(v.end(), {d.parent, d.nfp, d.nchild, d.child[0], d.child[1], d.nfc[0], d.nfc[1], d.kc[0], d.kc[1],
                           d.map[0], d.map[1]});
      break;
    case CL_TABLE_GATHER:
      for (const auto& d : p.gather) v.insert(v.end(), {d.child, d.parent, d.nfc, d.kc, d.nfp, d.rs, d.map});
      break;
    case CL_TABLE_MAPS:
      v.assign(p.maps.begin(), p.maps.end());
      break;
    case CL_TABLE_OFF:
      v.assign(p.off_all.begin(), p.off_all.end());
      break;
    case CL_TABLE_LD:
      v.assign(p.ld_all.begin(), p.ld_all.end());
      break;
  }
  *count = (long long)v.size();
  if (!out) return CL_OK;
  if (cap < (long long)v.size()) return CL_ERR_INVALID_ARG;
  std::copy(v.begin(), v.end(), out);
  return CL_OK;
}

int cl_plan_get_node(const cl_plan* plan, int i, int* parent, int* level, int* n_sep, int* n_bnd, int* sep,
                     int* bnd) {
  if (plan && plan->p.ragged) return CL_ERR_UNSUPPORTED;
  if (!plan || i < 0 || i >= (int)plan->p.nodes.size()) return CL_ERR_INVALID_ARG;
  const cl::SNode& n = plan->p.nodes[i];
  if (parent) *parent = n.parent;
  if (level) *level = n.level;
  if (n_sep) *n_sep = (int)n.sep.size();
  if (n_bnd) *n_bnd = (int)n.bnd.size();
  if (sep) std::memcpy(sep, n.sep.data(), n.sep.size() * sizeof(int));
  if (bnd) std::memcpy(bnd, n.bnd.data(), n.bnd.size() * sizeof(int));
  return CL_OK;
}

static void prof_clear(Plan& p) {
  for (auto& r : p.prof) {
    cudaEventDestroy((cudaEvent_t)r.ev0);
    cudaEventDestroy((cudaEvent_t)r.ev1);
  }
  p.prof.clear();
}

int cl_profile_enable(cl_plan* plan, int enable) {
  if (!compute_ready(plan)) return CL_ERR_INVALID_ARG;
  prof_clear(plan->p);
  plan->p.profiling = enable != 0;
  return CL_OK;
}

int cl_profile_read(cl_plan* plan, cl_profile_entry* out, int cap, int* n) {
  if (!compute_ready(plan) || !n || (cap > 0 && !out)) return CL_ERR_INVALID_ARG;
  cl_profile_entry acc[cl::F_COUNT];
  std::memset(acc, 0, sizeof(acc));
  for (auto& r : plan->p.prof) {
    cudaError_t e = cudaEventSynchronize((cudaEvent_t)r.ev1);
    if (e != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, (cudaEvent_t)r.ev0, (cudaEvent_t)r.ev1);
    cl_profile_entry& a = acc[r.family];
    a.launches += 1;
    a.total_ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
  }
  int k = 0;
  for (int f = 0; f < cl::F_COUNT; ++f) {
    if (acc[f].launches == 0) continue;
    if (k < cap) {
      out[k] = acc[f];
      std::strncpy(out[k].name, kFamilyName[f], sizeof(out[k].name) - 1);
    }
    ++k;
  }
  *n = k;
  return CL_OK;
}

int cl_profile_trace(cl_plan* plan, cl_trace_entry* out, int cap, int* n) {
  if (!compute_ready(plan) || !n || (cap > 0 && !out)) return CL_ERR_INVALID_ARG;
  const auto& recs = plan->p.prof;
  for (auto& r : recs) {
    cudaError_t e = cudaEventSynchronize((cudaEvent_t)r.ev1);
    if (e != cudaSuccess) return cuda_status(e);
  }
  *n = (int)recs.size();
  for (size_t i = 0; i < recs.size() && (int)i < cap; ++i) {
    const auto& r = recs[i];
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, (cudaEvent_t)recs[0].ev0, (cudaEvent_t)r.ev0);
    cudaEventElapsedTime(&b, (cudaEvent_t)recs[0].ev0, (cudaEvent_t)r.ev1);
    cl_trace_entry& t = out[i];
    std::memset(&t, 0, sizeof(t));
    std::strncpy(t.name, kFamilyName[r.family], sizeof(t.name) - 1);
    t.phase = r.phase;
    t.op = r.op;
    t.stream = r.stream;
    t.level = r.level;
    t.t0_us = 1e3 * a;
    t.t1_us = 1e3 * b;
  }
  return CL_OK;
}

void cl_destroy_plan(cl_plan* plan) {
  if (!plan) return;
  prof_clear(plan->p);
  free_device(plan->p);
  delete plan;
}

const char* cl_error_string(int status) {
  switch (status) {
    case CL_OK: return "success";
    case CL_ERR_INVALID_ARG: return "invalid argument";
    case CL_ERR_OOM: return "out of device memory";
    case CL_ERR_CUDA: return "CUDA error";
    case CL_ERR_SINGULAR: return "singular or near-singular pivot block";
    case CL_ERR_NONFINITE: return "non-finite result";
    case CL_ERR_TIMEOUT: return "device wait timed out";
    case CL_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

}  // extern "C"
