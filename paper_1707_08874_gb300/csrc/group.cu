// Groups of plans: several lattice shapes (each with its own batch of
// replicas) evaluated side by side on forked streams, and the whole fixed
// schedule captured once into a CUDA graph and replayed with one launch.
#include <vector>

#include "clselinv.h"

struct cl_group {
  std::vector<cl_plan*> plans;  // not owned
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (the legacy default stream cannot be captured)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return CL_OK;
  return e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA;
}

void release(cl_group* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (auto s : g->streams) cudaStreamDestroy(s);
  for (auto e : g->join) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->cap) cudaStreamDestroy(g->cap);
  g->cap = nullptr;
  g->exec = nullptr;
  g->graph = nullptr;
}

}  // namespace

extern "C" {

int cl_group_create(int nplans, cl_plan* const* plans, cl_group** out) {
  if (!out || nplans < 1 || !plans) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  cl_group* g = new cl_group();
  cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  for (int i = 0; i < nplans && e == cudaSuccess; ++i) {
    if (!plans[i]) e = cudaErrorInvalidValue;
    g->plans.push_back(plans[i]);
    cudaStream_t s = nullptr;
    cudaEvent_t j = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (s) g->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (j) g->join.push_back(j);
  }
  if (e != cudaSuccess) {
    release(g);
    delete g;
    return e == cudaErrorInvalidValue ? CL_ERR_INVALID_ARG : status_of(e);
  }
  *out = g;
  return CL_OK;
}

int cl_group_drift_eval(cl_group* g, const double* const* links, double m, double mu, double nf,
                        double* const* Gfwd, double* const* Gbwd, double* const* Kf, cudaStream_t stream) {
  if (!g || !links || !Gfwd || !Gbwd || !Kf) return CL_ERR_INVALID_ARG;
  cudaError_t e = cudaEventRecord(g->fork, stream);
  if (e != cudaSuccess) return status_of(e);
  const int n = (int)g->plans.size();
  for (int i = 0; i < n; ++i) {
    if ((e = cudaStreamWaitEvent(g->streams[i], g->fork, 0)) != cudaSuccess) return status_of(e);
    const int st = cl_drift_eval(g->plans[i], links[i], m, mu, nf, nullptr, Gfwd[i], Gbwd[i], Kf[i], g->streams[i]);
    if (st != CL_OK) return st;
    if ((e = cudaEventRecord(g->join[i], g->streams[i])) != cudaSuccess) return status_of(e);
    if ((e = cudaStreamWaitEvent(stream, g->join[i], 0)) != cudaSuccess) return status_of(e);
  }
  return CL_OK;
}

int cl_group_capture(cl_group* g, const double* const* links, double m, double mu, double nf, double* const* Gfwd,
                     double* const* Gbwd, double* const* Kf, cudaStream_t stream) {
  if (!g) return CL_ERR_INVALID_ARG;
  // capture on the group's own stream (capture executes nothing, so no
  // ordering with `stream` is needed; the legacy default stream cannot be
  // captured)
  (void)stream;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return status_of(e);
  const int st = cl_group_drift_eval(g, links, m, mu, nf, Gfwd, Gbwd, Kf, g->cap);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->cap, &graph);
  if (st != CL_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return status_of(e);
  g->graph = graph;
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  return status_of(e);
}

int cl_group_launch(cl_group* g, cudaStream_t stream) {
  if (!g || !g->exec) return CL_ERR_INVALID_ARG;
  return status_of(cudaGraphLaunch(g->exec, stream));
}

void cl_group_destroy(cl_group* g) {
  if (!g) return;
  release(g);
  delete g;
}

}  // extern "C"
