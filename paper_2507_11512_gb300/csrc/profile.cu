// Per-kernel-class timing with CUDA events (tracing of the solve's motifs:
// SpMV, Gauss-Seidel, restriction, prolongation, CGS2, ...).  Each profiled
// launch is bracketed by two events recorded on the launch's own stream; the
// report sums the elapsed times and the algorithmic DRAM bytes per class and
// level.  Disabled by default; costs nothing when disabled.

#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "hpg_internal.cuh"

namespace hpg {

struct ProfRec {
  int cls, level, prec;
  double bytes;
  int ev;   // index of the start event; ev + 1 is the stop event
};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> events;
  size_t used = 0;
  std::vector<ProfRec> recs;
};

static const char* kNames[K_NUM_CLASSES] = {
    "gen_ell",      "permute",         "spmv",        "residual_fp64", "gs_colour_phase",
    "restrict",     "prolong",         "cgs2_gemvt",  "cgs2_reorth",   "cgs2_final_givens",
    "arnoldi_scale", "trsm",           "basis_combine", "update_x",    "cycle_start",
    "norm",         "vcycle_coarse_cluster", "diag_scale_gradient"};

const char* kernel_class_name(int cls) {
  return (cls >= 0 && cls < K_NUM_CLASSES) ? kNames[cls] : "unknown";
}

int prof_begin(hpg_problem* h, cudaStream_t s) {
  Profiler* p = h->prof;
  if (!p || !p->on) return -1;
  while (p->events.size() < p->used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p->events.push_back(e);
  }
  const int slot = (int)p->used;
  p->used += 2;
  cudaEventRecord(p->events[slot], s);
  return slot;
}

void prof_end(hpg_problem* h, int slot, int cls, int level, int prec, double bytes,
              cudaStream_t s) {
  if (slot < 0) return;
  Profiler* p = h->prof;
  cudaEventRecord(p->events[slot + 1], s);
  p->recs.push_back(ProfRec{cls, level, prec, bytes, slot});
}

void destroy_profiler(hpg_problem* h) {
  if (!h->prof) return;
  for (cudaEvent_t e : h->prof->events) cudaEventDestroy(e);
  delete h->prof;
  h->prof = nullptr;
}

}  // namespace hpg

using namespace hpg;

extern "C" {

HPG_API int hpg_set_profiling(hpg_problem_t* h, int enable) {
  if (!h) {
    set_error("hpg_set_profiling: NULL handle");
    return HPG_ERR_INVALID;
  }
  if (!h->prof) h->prof = new Profiler();
  h->prof->on = enable != 0;
  h->profiling = enable != 0;
  h->prof->used = 0;
  h->prof->recs.clear();
  return HPG_OK;
}

HPG_API int hpg_profile_report(hpg_problem_t* h, hpg_kernel_stat* out, int capacity,
                               int* count) {
  if (!h || !count || (capacity > 0 && !out)) {
    set_error("hpg_profile_report: invalid argument");
    return HPG_ERR_INVALID;
  }
  *count = 0;
  if (!h->prof) return HPG_OK;
  Profiler* p = h->prof;
  std::map<std::tuple<int, int, int>, hpg_kernel_stat> agg;
  for (const ProfRec& r : p->recs) {
    HPG_CK(cudaEventSynchronize(p->events[r.ev + 1]));
    float ms = 0.f;
    HPG_CK(cudaEventElapsedTime(&ms, p->events[r.ev], p->events[r.ev + 1]));
    hpg_kernel_stat& st = agg[std::make_tuple(r.cls, r.level, r.prec)];
    st.name = kernel_class_name(r.cls);
    st.level = r.level;
    st.prec = r.prec;
    st.launches += 1;
    st.total_ms += ms;
    st.bytes += r.bytes;
  }
  int n = 0;
  for (auto& kv : agg) {
    if (n < capacity) out[n] = kv.second;
    n++;
  }
  *count = n;
  p->used = 0;
  p->recs.clear();
  return HPG_OK;
}

}  // extern "C"
