// api.cu -- the C ABI declared in include/bsparareal.h.
//
// Host code here validates arguments, owns the device memory of the handles
// and enqueues kernels; every step of the numerical path runs in the kernels
// of solver.cu and pinn.cu.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bsparareal.h"
#include "bs_common.cuh"
#include "bs_internal.h"

using bsp::Inst;

namespace {

struct Class {
  int M = 0, NW = 0, C = 1, maxP = 0;
  int s2 = 1;  // slices per CTA of the fine propagation (2: instances' slices in pairs)
  std::vector<int32_t> ids;
  int32_t* d_ids = nullptr;
};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// NVTX range over a scope: the phases of a call appear in profilers that
// record NVTX (ncu --nvtx); without a tool attached a range costs a check of a
// function pointer.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return BS_OK;
  if (e == cudaErrorMemoryAllocation) return BS_ENOMEM;
  return BS_ECUDA;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Partition of the Nx-1 rows (interior + Dirichlet row at Smax) over a
// cluster of C CTAs x NW warps x 32 lanes x M rows.  cl_target is the number of
// SMs one grid may occupy: the problem's slices share the 148 SMs, so few
// slices spread each grid over a cluster of several CTAs (several SMs), many
// slices keep one CTA per grid.  Grids above 4096 rows need a cluster.
bool choose_partition(int Nx, int cl_target, int* M, int* NW, int* C) {
  const int rows = Nx - 1;
  if (rows <= 4096 && (cl_target <= 1 || rows < 2 * 4 * 32 * 2)) {
    *C = 1;
    if (rows <= 64) { *NW = 1; *M = 2; return true; }
    if (rows <= 128) { *NW = 2; *M = 2; return true; }
    *NW = 4;
    int m = 2;
    while (m * 128 < rows) m *= 2;
    *M = m;
    return true;
  }
  int c = 1;
  while (c < cl_target && c < 16) c *= 2;
  while (c * 4 * 32 * 2 > 2 * rows && c > 1) c /= 2;  // at most half of the rows padding
  while (c * 4 * 32 * 32 < rows && c < 16) c *= 2;  // at most 32 rows per thread
  for (; c >= 1; c /= 2) {
    int m = 2;
    while (m * 128 * c < rows && m < 32) m *= 2;
    if (m * 128 * c < rows) return false;
    if (bsp::partition_supported(m, 4, c)) {
      *C = c;
      *NW = 4;
      *M = m;
      return true;
    }
  }
  return false;
}

// SMs per grid from the number of slices that run at once (148 SMs), or the
// BSP_CLUSTER environment variable (1, 2, 4, 8 or 16) when set.
int cluster_target(const bs_params* p, int n) {
  if (const char* env = getenv("BSP_CLUSTER")) {
    const int v = atoi(env);
    if (v >= 1 && v <= 16) return v;
  }
  int64_t slices = 0;
  for (int i = 0; i < n; ++i) slices += p[i].P;
  int c = 1;
  while (c < 16 && slices * (2 * c) <= 148) c *= 2;
  return c;
}

struct Part {
  int M, NW, C;
  int s2 = 1;
};

// Every compiled partition that holds an Nx-point grid with at most half of
// its rows padding.
std::vector<Part> candidate_partitions(int Nx) {
  std::vector<Part> out;
  const int rows = Nx - 1;
  for (int C = 1; C <= 16; C *= 2)
    for (int NW = 1; NW <= 8; NW *= 2)
      for (int M = 2; M <= 32; M *= 2) {
        const int64_t R = (int64_t)M * NW * 32 * C;
        if (R >= rows && 2 * (R - rows) <= R && bsp::partition_supported(M, NW, C)) {
          out.push_back(Part{M, NW, C, 1});
          if (bsp::s2_supported(M, NW, C)) out.push_back(Part{M, NW, C, 2});
        }
      }
  return out;
}

int validate(const bs_params* p, int32_t n_instances) {
  for (int i = 0; i < n_instances; ++i) {
    const bs_params& q = p[i];
    if (!finite_pos(q.K) || !finite_pos(q.sigma) || !std::isfinite(q.r) || q.r < 0.0 || !finite_pos(q.T) ||
        !finite_pos(q.Smax) || !(q.Smax > q.K) || q.Nx < 5 || q.P < 1 || q.fine_steps < 1 || q.coarse_steps < 1)
      return BS_EINVAL;
  }
  return BS_OK;
}

}  // namespace

static int problem_create(const bs_params* p, int32_t n_instances, const Part* parts, bs_problem** out);

struct bs_problem {
  int n_inst = 0;
  std::vector<Inst> h_insts;
  Inst* d_insts = nullptr;
  double* pool = nullptr;
  double* exptab = nullptr;
  std::vector<Class> classes;
  int64_t total_state = 0, total_slice = 0, total_tasks = 0, total_tasks1 = 0, total_norm = 0;
  int maxP = 0;
  // Parareal workspace (allocated on first use)
  double *buf0 = nullptr, *buf1 = nullptr, *fbuf = nullptr, *gold = nullptr, *gtab = nullptr, *normbuf = nullptr;
  double* Xgrid = nullptr;
  int xgrid_din = 0;
  double* norms_dev = nullptr;
  int norms_cap = 0;
  bsp::Ctrl* ctrl = nullptr;
  int* d_status = nullptr;  // BS_TIMEOUT once a bounded exchange wait gave up
  // per solve, zeroed at its start: the fine launches' task counters
  // [(maxP + 1) x classes, iteration k at row k + 1] and the count of instances
  // still iterating after iteration k [maxP]
  int* d_sched = nullptr;
  int64_t sched_n = 0;
};

struct pinn_model {
  bsp::MlpDev dev{};
  int64_t n_params = 0;
  double* p64 = nullptr;
  float* p32 = nullptr;
  double* mom1 = nullptr;
  double* mom2 = nullptr;
  double* grad = nullptr;
  double* loss3 = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int step = 0;
  unsigned char* tc_packed = nullptr;
  int* status = nullptr;
};

extern "C" {

const char* bs_status_string(int status) {
  switch (status) {
    case BS_OK: return "ok";
    case BS_EINVAL: return "invalid argument";
    case BS_ECUDA: return "CUDA error";
    case BS_ENOMEM: return "out of memory";
    case BS_NOT_CONVERGED: return "not converged";
    case BS_DIVERGED: return "diverged (non-finite norm)";
    case BS_TIMEOUT: return "timeout";
    case BS_EUNSUPPORTED: return "unsupported size or mode";
  }
  return "unknown status";
}

const char* bs_version(void) { return "bsparareal 0.1 sm_103a"; }

void bs_problem_destroy(bs_problem* prob) {
  if (!prob) return;
  cudaFree(prob->d_insts);
  cudaFree(prob->pool);
  cudaFree(prob->exptab);
  for (auto& c : prob->classes) cudaFree(c.d_ids);
  cudaFree(prob->buf0);
  cudaFree(prob->buf1);
  cudaFree(prob->fbuf);
  cudaFree(prob->gold);
  cudaFree(prob->gtab);
  cudaFree(prob->normbuf);
  cudaFree(prob->Xgrid);
  cudaFree(prob->norms_dev);
  cudaFree(prob->ctrl);
  cudaFree(prob->d_status);
  cudaFree(prob->d_sched);
  delete prob;
}

}  // extern "C"

// The handle for given partitions (one per instance): device tables, set-up kernels.
static int problem_create(const bs_params* p, int32_t n_instances, const Part* parts, bs_problem** out) {
  *out = nullptr;
  bs_problem* prob = new (std::nothrow) bs_problem();
  if (!prob) return BS_ENOMEM;
  prob->n_inst = n_instances;
  prob->h_insts.resize(n_instances);
  int64_t coef = 0, ex = 0;
  for (int i = 0; i < n_instances; ++i) {
    const bs_params& q = p[i];
    Inst in{};
    in.K = q.K;
    in.sigma = q.sigma;
    in.r = q.r;
    in.T = q.T;
    in.Smax = q.Smax;
    in.dS = q.Smax / (double)(q.Nx - 1);
    in.Nx = q.Nx;
    in.P = q.P;
    in.Mf = q.fine_steps;
    in.Mg = q.coarse_steps;
    in.M = parts[i].M;
    in.NW = parts[i].NW;
    in.C = parts[i].C;
    in.Ws = in.C * in.NW;
    in.R = in.Ws * 32 * in.M;
    in.Np = in.R - (q.Nx - 1);
    const int64_t bs = bsp::coef_block_size(in.M, in.Ws * 32, in.Ws);
    in.coef_cn = coef;
    coef += bs;
    in.coef_ie = coef;
    coef += bs;
    in.exp_cn = ex;
    ex += q.fine_steps + 1;
    in.exp_ie = ex;
    ex += q.coarse_steps + 1;
    in.exp_sl = ex;
    ex += q.P + 1;
    in.state_off = prob->total_state;
    prob->total_state += (int64_t)(q.P + 1) * q.Nx;
    in.slice_off = prob->total_slice;
    prob->total_slice += (int64_t)q.P * q.Nx;
    in.task_off = prob->total_tasks;
    prob->total_tasks += q.P;
    in.task1_off = prob->total_tasks1;
    prob->total_tasks1 += q.P + 1;
    in.norm_off = prob->total_norm;
    prob->total_norm += (int64_t)(q.P + 1) * in.C;
    if (q.P > prob->maxP) prob->maxP = q.P;
    prob->h_insts[i] = in;
    Class* cl = nullptr;
    for (auto& c : prob->classes)
      if (c.M == in.M && c.NW == in.NW && c.C == in.C && c.s2 == parts[i].s2) cl = &c;
    if (!cl) {
      prob->classes.push_back(Class{});
      cl = &prob->classes.back();
      cl->M = in.M;
      cl->NW = in.NW;
      cl->C = in.C;
      cl->s2 = parts[i].s2;
    }
    cl->ids.push_back(i);
    if (q.P > cl->maxP) cl->maxP = q.P;
  }
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&prob->d_insts, n_instances)) != cudaSuccess ||
      (e = dalloc(&prob->pool, (size_t)coef)) != cudaSuccess || (e = dalloc(&prob->exptab, (size_t)ex)) != cudaSuccess ||
      (e = dalloc(&prob->d_status, 1)) != cudaSuccess || (e = cudaMemset(prob->d_status, 0, sizeof(int))) != cudaSuccess) {
    bs_problem_destroy(prob);
    return map_err(e);
  }
  prob->sched_n = (int64_t)(prob->maxP + 1) * (int64_t)prob->classes.size() + prob->maxP;
  if ((e = dalloc(&prob->d_sched, (size_t)prob->sched_n)) != cudaSuccess) {
    bs_problem_destroy(prob);
    return map_err(e);
  }
  e = cudaMemcpy(prob->d_insts, prob->h_insts.data(), sizeof(Inst) * n_instances, cudaMemcpyHostToDevice);
  for (auto& c : prob->classes) {
    if (e == cudaSuccess) e = dalloc(&c.d_ids, c.ids.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(c.d_ids, c.ids.data(), sizeof(int32_t) * c.ids.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = bsp::launch_setup(prob->d_insts, c.d_ids, (int)c.ids.size(), c.NW * c.C, prob->pool, prob->exptab, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    bs_problem_destroy(prob);
    return map_err(e);
  }
  *out = prob;
  return BS_OK;
}

extern "C" {

int bs_problem_init(const bs_params* p, int32_t n_instances, bs_problem** out) {
  Range range_("bs_problem_init");
  if (!p || !out || n_instances <= 0) return BS_EINVAL;
  *out = nullptr;
  if (validate(p, n_instances) != BS_OK) return BS_EINVAL;
  const int cl_target = cluster_target(p, n_instances);
  std::vector<Part> parts(n_instances);
  Part forced{0, 0, 0, 1};
  if (const char* env = getenv("BSP_PARTITION")) {  // "M,NW,C" or "M,NW,C,S2" for every instance
    const int got = sscanf(env, "%d,%d,%d,%d", &forced.M, &forced.NW, &forced.C, &forced.s2);
    if (got < 3 || !bsp::partition_supported(forced.M, forced.NW, forced.C)) return BS_EUNSUPPORTED;
    if (got < 4) forced.s2 = 1;
    if (forced.s2 != 1 && !(forced.s2 == 2 && bsp::s2_supported(forced.M, forced.NW, forced.C)))
      return BS_EUNSUPPORTED;
  }
  for (int i = 0; i < n_instances; ++i) {
    if (forced.M > 0) {
      if ((int64_t)forced.M * forced.NW * 32 * forced.C < p[i].Nx - 1) return BS_EUNSUPPORTED;
      parts[i] = forced;
    } else if (!choose_partition(p[i].Nx, cl_target, &parts[i].M, &parts[i].NW, &parts[i].C)) {
      return BS_EUNSUPPORTED;
    }
  }
  if (forced.M == 0) {
    // slice pairs where the class supports them and has slices enough to keep
    // every cluster busy twice over (throughput rather than latency); on one-CTA
    // grids only with 32 rows per thread, where one slice per CTA leaves one
    // warp per sub-partition (16 rows fit two CTAs per SM already);
    // BSP_S2 = 1 or 2 decides instead
    int s2_env = 0;
    if (const char* env = getenv("BSP_S2")) s2_env = atoi(env);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < n_instances; ++i) {
      Part& q = parts[i];
      if (!bsp::s2_supported(q.M, q.NW, q.C) || (q.C == 1 && q.M < 32 && !s2_env)) continue;
      int64_t slices = 0;
      for (int j = 0; j < n_instances; ++j)
        if (parts[j].M == q.M && parts[j].NW == q.NW && parts[j].C == q.C) slices += p[j].P;
      const bool pairs = s2_env ? s2_env == 2 : slices >= 2 * (int64_t)(nsm / q.C);
      q.s2 = pairs ? 2 : 1;
    }
  }
  return problem_create(p, n_instances, parts.data(), out);
}

// Device time of one fine_propagate over the instances `sub` (all with the
// partition `part`) on zero states, best of two runs after one warm-up run.
static int time_partition(const std::vector<bs_params>& sub, Part part, float* ms) {
  std::vector<Part> parts(sub.size(), part);
  bs_problem* pr = nullptr;
  int rc = problem_create(sub.data(), (int32_t)sub.size(), parts.data(), &pr);
  if (rc != BS_OK) return rc;
  double *a = nullptr, *b = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = dalloc(&a, pr->total_slice);
  if (e == cudaSuccess) e = dalloc(&b, pr->total_slice);
  if (e == cudaSuccess) e = cudaMemset(a, 0, sizeof(double) * pr->total_slice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int run = 0; run < 3 && e == cudaSuccess && rc == BS_OK; ++run) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) rc = fine_propagate(pr, a, b, nullptr, nullptr);
    if (e == cudaSuccess && rc == BS_OK) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess && rc == BS_OK) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess && rc == BS_OK) e = cudaEventElapsedTime(&t, e0, e1);
    if (run == 1 || (run == 2 && t < best)) best = t;
  }
  if (rc == BS_OK && e == cudaSuccess) {
    int st = 0;
    e = cudaMemcpy(&st, pr->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && st != 0) rc = BS_TIMEOUT;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  bs_problem_destroy(pr);
  if (rc == BS_OK && e != cudaSuccess) rc = map_err(e);
  *ms = best;
  return rc;
}

int bs_problem_init_tuned(const bs_params* p, int32_t n_instances, bs_problem** out, bs_tuning* report,
                          int32_t report_cap, int32_t* n_report) {
  Range range_("bs_problem_init_tuned");
  if (!p || !out || n_instances <= 0 || (report_cap > 0 && !report)) return BS_EINVAL;
  *out = nullptr;
  if (n_report) *n_report = 0;
  if (validate(p, n_instances) != BS_OK) return BS_EINVAL;
  std::vector<Part> parts(n_instances);
  std::vector<int> done(n_instances, 0);
  int32_t nr = 0;
  for (int i0 = 0; i0 < n_instances; ++i0) {
    if (done[i0]) continue;
    const int Nx = p[i0].Nx;
    const std::vector<Part> cand = candidate_partitions(Nx);
    if (cand.empty()) return BS_EUNSUPPORTED;
    // tuning subset: instances of this grid size, enough for >= 4096 slices
    std::vector<int> group;
    for (int i = i0; i < n_instances; ++i)
      if (p[i].Nx == Nx) group.push_back(i);
    std::vector<bs_params> sub;
    int64_t slices = 0;
    for (int i : group) {
      if (slices >= 4096) break;
      bs_params q = p[i];
      if (q.fine_steps > 128) q.fine_steps = 128;
      q.coarse_steps = 1;
      sub.push_back(q);
      slices += q.P;
    }
    Part best = cand[0];
    float best_ms = -1.0f;
    for (const Part& c : cand) {
      float ms = 0.0f;
      const int rc = time_partition(sub, c, &ms);
      if (rc == BS_TIMEOUT) return rc;
      if (rc != BS_OK) {  // this candidate does not fit (memory, launch resources)
        (void)cudaGetLastError();
        continue;
      }
      if (nr < report_cap) report[nr] = bs_tuning{Nx, c.M, c.NW, c.C, c.s2, ms, 0};
      ++nr;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (best_ms < 0.0f) return BS_EUNSUPPORTED;
    for (int k = 0; k < (nr < report_cap ? nr : report_cap); ++k)
      if (report[k].Nx == Nx)
        report[k].chosen = (report[k].M == best.M && report[k].NW == best.NW && report[k].C == best.C &&
                            report[k].S2 == best.s2);
    for (int i : group) {
      parts[i] = best;
      done[i] = 1;
    }
  }
  if (n_report) *n_report = nr;
  return problem_create(p, n_instances, parts.data(), out);
}

int bs_problem_init_partitioned(const bs_params* p, int32_t n_instances, const bs_tuning* parts_in,
                                int32_t n_parts, bs_problem** out) {
  Range range_("bs_problem_init_partitioned");
  if (!p || !out || n_instances <= 0 || !parts_in || n_parts <= 0) return BS_EINVAL;
  *out = nullptr;
  if (validate(p, n_instances) != BS_OK) return BS_EINVAL;
  std::vector<Part> parts(n_instances);
  for (int i = 0; i < n_instances; ++i) {
    const bs_tuning* hit = nullptr;
    for (int k = 0; k < n_parts && !hit; ++k)
      if (parts_in[k].Nx == p[i].Nx && parts_in[k].chosen) hit = &parts_in[k];
    if (!hit) return BS_EINVAL;  // no partition given for this grid size
    const Part c{hit->M, hit->NW, hit->C, hit->S2};
    if (!bsp::partition_supported(c.M, c.NW, c.C) ||
        (c.s2 != 1 && !(c.s2 == 2 && bsp::s2_supported(c.M, c.NW, c.C))) ||
        (int64_t)c.M * c.NW * 32 * c.C < p[i].Nx - 1)
      return BS_EUNSUPPORTED;
    parts[i] = c;
  }
  return problem_create(p, n_instances, parts.data(), out);
}

int bs_problem_info(const bs_problem* prob, int32_t* n_instances, int64_t* total_state_doubles,
                    int64_t* total_slice_doubles) {
  if (!prob) return BS_EINVAL;
  if (n_instances) *n_instances = prob->n_inst;
  if (total_state_doubles) *total_state_doubles = prob->total_state;
  if (total_slice_doubles) *total_slice_doubles = prob->total_slice;
  return BS_OK;
}

int bs_problem_device_status(const bs_problem* prob, int* status) {
  if (!prob || !status) return BS_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, prob->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  return map_err(e);
}

int bs_problem_slices_per_cta(const bs_problem* prob, int32_t i, int32_t* s2) {
  if (!prob || !s2 || i < 0 || i >= prob->n_inst) return BS_EINVAL;
  *s2 = 1;
  const Inst& in = prob->h_insts[i];
  for (const auto& c : prob->classes)
    if (c.M == in.M && c.NW == in.NW && c.C == in.C)
      for (int32_t id : c.ids)
        if (id == i) *s2 = c.s2;
  return BS_OK;
}

int bs_problem_partition(const bs_problem* prob, int32_t i, int32_t* M, int32_t* NW, int32_t* C) {
  if (!prob || i < 0 || i >= prob->n_inst) return BS_EINVAL;
  if (M) *M = prob->h_insts[i].M;
  if (NW) *NW = prob->h_insts[i].NW;
  if (C) *C = prob->h_insts[i].C;
  return BS_OK;
}

static int propagate(bs_problem* prob, bool cn, const double* U_in, double* U_out, const uint8_t* active,
                     void* stream) {
  if (!prob || !U_in || !U_out) return BS_EINVAL;
  if (((uintptr_t)U_in | (uintptr_t)U_out) & 15) return BS_EINVAL;
  const double* ie = U_in + prob->total_slice;
  const double* oe = U_out + prob->total_slice;
  if (U_in < oe && U_out < ie) return BS_EINVAL;  // overlap
  cudaStream_t s = (cudaStream_t)stream;
  for (auto& c : prob->classes) {
    bsp::PropArgs a{};
    a.insts = prob->d_insts;
    a.ids = c.d_ids;
    a.pool = prob->pool;
    a.exptab = prob->exptab;
    a.in = U_in;
    a.out = U_out;
    a.in_state = 0;
    a.out_state = 0;
    a.mode = bsp::PropArgs::kPlain;
    a.k_iter = -1;
    a.active = active;
    a.status = prob->d_status;
    cudaError_t e = bsp::launch_prop(c.M, c.NW, c.C, c.s2, cn, a, (int)c.ids.size(), c.maxP, s);
    if (e != cudaSuccess) return map_err(e);
  }
  return BS_OK;
}

int fine_propagate(bs_problem* prob, const double* U_in, double* U_out, const uint8_t* active, void* stream) {
  Range range_("fine_propagate");
  return propagate(prob, true, U_in, U_out, active, stream);
}

int coarse_propagate(bs_problem* prob, const double* U_in, double* U_out, const uint8_t* active, void* stream) {
  Range range_("coarse_propagate");
  return propagate(prob, false, U_in, U_out, active, stream);
}

int serial_fine(bs_problem* prob, double* U_out, void* stream) {
  Range range_("serial_fine");
  if (!prob || !U_out || ((uintptr_t)U_out & 15)) return BS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  for (auto& c : prob->classes) {
    bsp::SerialArgs a{prob->d_insts, c.d_ids, prob->pool, prob->exptab, U_out, prob->d_status};
    cudaError_t e = bsp::launch_serial(c.M, c.NW, c.C, a, (int)c.ids.size(), s);
    if (e != cudaSuccess) return map_err(e);
  }
  return BS_OK;
}

// ---------------------------------------------------------------------------
// Network handles
// ---------------------------------------------------------------------------

// SplitMix64 (Steele, Lea, Flood 2014): output number i+1 of the sequence whose state starts at `seed`.
static uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

void pinn_destroy(pinn_model* m) {
  if (!m) return;
  cudaFree(m->p64);
  cudaFree(m->p32);
  cudaFree(m->mom1);
  cudaFree(m->mom2);
  cudaFree(m->grad);
  cudaFree(m->loss3);
  cudaFree(m->ws);
  cudaFree(m->tc_packed);
  cudaFree(m->status);
  delete m;
}

static int upload_params(pinn_model* m, const double* host) {
  cudaError_t e = cudaMemcpy(m->p64, host, sizeof(double) * m->n_params, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = bsp::launch_f64_to_f32(m->p64, m->p32, m->n_params, 0);
  if (e == cudaSuccess) e = cudaMemset(m->mom1, 0, sizeof(double) * m->n_params);
  if (e == cudaSuccess) e = cudaMemset(m->mom2, 0, sizeof(double) * m->n_params);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  m->step = 0;
  return map_err(e);
}

int pinn_create(const int32_t* widths, int32_t n_layers, const double* in_lo, const double* in_hi, uint64_t seed,
                pinn_model** out) {
  if (!widths || !out || !in_lo || !in_hi || n_layers < 1 || n_layers > 15) return BS_EINVAL;
  *out = nullptr;
  const int d_in = widths[0];
  if (!(d_in == 2 || d_in == 5) || widths[n_layers] != 1) return BS_EINVAL;
  int max_w = 0;
  for (int l = 0; l <= n_layers; ++l) {
    if (widths[l] < 1 || widths[l] > 256) return BS_EINVAL;
    if (widths[l] > max_w) max_w = widths[l];
  }
  for (int i = 0; i < d_in; ++i)
    if (!std::isfinite(in_lo[i]) || !std::isfinite(in_hi[i]) || !(in_hi[i] > in_lo[i])) return BS_EINVAL;
  pinn_model* m = new (std::nothrow) pinn_model();
  if (!m) return BS_ENOMEM;
  m->dev.n_lin = n_layers;
  m->dev.d_in = d_in;
  m->dev.max_w = max_w;
  int64_t off = 0;
  for (int l = 0; l <= n_layers; ++l) m->dev.widths[l] = widths[l];
  for (int l = 1; l <= n_layers; ++l) {
    m->dev.poff[l] = off;
    off += (int64_t)widths[l] * widths[l - 1] + widths[l];
  }
  for (int i = 0; i < d_in; ++i) {
    m->dev.lo[i] = in_lo[i];
    m->dev.hi[i] = in_hi[i];
  }
  m->n_params = off;
  cudaError_t e;
  if ((e = dalloc(&m->p64, off)) != cudaSuccess || (e = dalloc(&m->p32, off)) != cudaSuccess ||
      (e = dalloc(&m->mom1, off)) != cudaSuccess || (e = dalloc(&m->mom2, off)) != cudaSuccess ||
      (e = dalloc(&m->grad, off)) != cudaSuccess || (e = dalloc(&m->loss3, 4)) != cudaSuccess) {
    pinn_destroy(m);
    return map_err(e);
  }
  m->dev.p64 = m->p64;
  m->dev.p32 = m->p32;
  if ((e = dalloc(&m->status, 1)) != cudaSuccess || (e = cudaMemset(m->status, 0, sizeof(int))) != cudaSuccess) {
    pinn_destroy(m);
    return map_err(e);
  }
  m->dev.status = m->status;
  if (bsp::tc_supported(m->dev)) {
    if ((e = dalloc(&m->tc_packed, bsp::tc_packed_bytes(m->dev) + 16)) != cudaSuccess) {
      pinn_destroy(m);
      return map_err(e);
    }
    m->dev.tc_packed = m->tc_packed;
  }
  // Xavier-uniform weights, zero biases
  std::vector<double> h(off, 0.0);
  for (int l = 1; l <= n_layers; ++l) {
    const double a = std::sqrt(6.0 / (double)(widths[l - 1] + widths[l]));
    const int64_t nw = (int64_t)widths[l] * widths[l - 1];
    for (int64_t q = 0; q < nw; ++q) {
      const int64_t idx = m->dev.poff[l] + q;
      const double u = (double)(splitmix64(seed, (uint64_t)idx) >> 11) * (1.0 / 9007199254740992.0);
      h[idx] = (2.0 * u - 1.0) * a;
    }
  }
  int rc = upload_params(m, h.data());
  if (rc != BS_OK) {
    pinn_destroy(m);
    return rc;
  }
  *out = m;
  return BS_OK;
}

int pinn_device_status(const pinn_model* m, int* status) {
  if (!m || !status) return BS_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, m->status, sizeof(int), cudaMemcpyDeviceToHost);
  return map_err(e);
}

int pinn_num_params(const pinn_model* m, int64_t* n) {
  if (!m || !n) return BS_EINVAL;
  *n = m->n_params;
  return BS_OK;
}

int pinn_set_weights(pinn_model* m, const double* flat_host) {
  if (!m || !flat_host) return BS_EINVAL;
  for (int64_t i = 0; i < m->n_params; ++i)
    if (!std::isfinite(flat_host[i])) return BS_EINVAL;
  return upload_params(m, flat_host);
}

int pinn_get_weights(const pinn_model* m, double* flat_host) {
  if (!m || !flat_host) return BS_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(flat_host, m->p64, sizeof(double) * m->n_params, cudaMemcpyDeviceToHost);
  return map_err(e);
}

int pinn_get_state(const pinn_model* m, double* theta, double* mom1, double* mom2, int64_t* step) {
  if (!m || !theta || !mom1 || !mom2 || !step) return BS_EINVAL;
  const size_t bytes = sizeof(double) * m->n_params;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(theta, m->p64, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(mom1, m->mom1, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(mom2, m->mom2, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) *step = m->step;
  return map_err(e);
}

int pinn_set_state(pinn_model* m, const double* theta, const double* mom1, const double* mom2, int64_t step) {
  if (!m || !theta || !mom1 || !mom2 || step < 0 || step > INT32_MAX) return BS_EINVAL;
  for (int64_t i = 0; i < m->n_params; ++i)
    if (!std::isfinite(theta[i]) || !std::isfinite(mom1[i]) || !std::isfinite(mom2[i]) || mom2[i] < 0.0)
      return BS_EINVAL;
  int rc = upload_params(m, theta);
  if (rc != BS_OK) return rc;
  const size_t bytes = sizeof(double) * m->n_params;
  cudaError_t e = cudaMemcpy(m->mom1, mom1, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->mom2, mom2, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) m->step = (int)step;
  return map_err(e);
}

int bs_wait_probe(int32_t arrive, int64_t limit_cycles, int32_t* status) {
  if (!status || limit_cycles < 1 || limit_cycles > (int64_t)1 << 34) return BS_EINVAL;
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return map_err(e);
  int h = -1;
  e = bsp::launch_wait_probe(arrive != 0, (long long)limit_cycles, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return map_err(e);
  *status = h;
  return BS_OK;
}

int pinn_eval(const pinn_model* m, int prec, const double* X, int64_t N, double* u, double* derivs, void* stream) {
  Range range_("pinn_eval");
  if (!m || N < 0 || prec < BS_FP64 || prec > BS_BF16) return BS_EINVAL;
  if (N == 0) return BS_OK;
  if (!X || !u || (((uintptr_t)X | (uintptr_t)u | (uintptr_t)derivs) & 15)) return BS_EINVAL;
  if (derivs && !(prec == BS_FP64 || prec == BS_FP32)) return BS_EINVAL;
  return map_err(bsp::launch_mlp_eval(m->dev, prec, X, N, u, derivs, (cudaStream_t)stream));
}

static int loss_grad_common(const pinn_model* mc, const double* X, const int8_t* kind, const double* y, int64_t N,
                            const bs_params* pp, double smax_over_K, int prec, double* loss3, double* grad,
                            cudaStream_t s) {
  pinn_model* m = const_cast<pinn_model*>(mc);
  if (!m || !X || !kind || !pp || N <= 0 || ((uintptr_t)y & 7)) return BS_EINVAL;
  if (prec < BS_FP64 || prec > BS_BF16) return BS_EINVAL;
  if (((uintptr_t)X & 15) || ((uintptr_t)grad & 7) || ((uintptr_t)loss3 & 7) || !std::isfinite(pp->K) ||
      !std::isfinite(pp->sigma) || !std::isfinite(pp->r) || !std::isfinite(pp->Smax) || !std::isfinite(smax_over_K))
    return BS_EINVAL;
  const size_t need = bsp::loss_grad_workspace_bytes(m->dev, N);
  if (need > m->ws_bytes) {
    cudaError_t e = cudaStreamSynchronize(s);  // the old workspace may still be in use
    if (e != cudaSuccess) return map_err(e);
    cudaFree(m->ws);
    m->ws = nullptr;
    m->ws_bytes = 0;
    e = cudaMalloc(&m->ws, need);
    if (e != cudaSuccess) return map_err(e);
    m->ws_bytes = need;
  }
  bsp::LossArgs la{X, kind, N, pp->K, pp->sigma, pp->r, pp->Smax, smax_over_K, prec, y};
  return map_err(bsp::launch_loss_grad(m->dev, la, loss3, grad, m->ws, m->ws_bytes, s));
}

int pinn_loss_grad(const pinn_model* m, const double* X, const int8_t* kind, int64_t N,
                   const bs_params* prob_params, double smax_over_K, int prec, double* loss3, double* grad,
                   void* stream) {
  Range range_("pinn_loss_grad");
  if (!loss3 || !grad) return BS_EINVAL;
  return loss_grad_common(m, X, kind, nullptr, N, prob_params, smax_over_K, prec, loss3, grad, (cudaStream_t)stream);
}

int pinn_loss_grad_data(const pinn_model* m, const double* X, const int8_t* kind, const double* y, int64_t N,
                        const bs_params* prob_params, double smax_over_K, int prec, double* loss3, double* grad,
                        void* stream) {
  Range range_("pinn_loss_grad_data");
  if (!loss3 || !grad || !y) return BS_EINVAL;
  return loss_grad_common(m, X, kind, y, N, prob_params, smax_over_K, prec, loss3, grad, (cudaStream_t)stream);
}

static int train_step_common(pinn_model* m, const double* X, const int8_t* kind, const double* y, int64_t N,
                             const bs_params* prob_params, double smax_over_K, int prec, double lr, double* loss3,
                             double* grad_out, void* stream) {
  if (!m || !std::isfinite(lr) || lr <= 0.0) return BS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  double* g = grad_out ? grad_out : m->grad;
  int rc = loss_grad_common(m, X, kind, y, N, prob_params, smax_over_K, prec, m->loss3, g, s);
  if (rc != BS_OK) return rc;
  m->step += 1;
  cudaError_t e = bsp::launch_adam(m->n_params, m->p64, m->mom1, m->mom2, g, m->step, lr, m->p32, s);
  if (e != cudaSuccess) return map_err(e);
  if (loss3) {
    int st = 0;
    e = cudaMemcpyAsync(loss3, m->loss3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, m->dev.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_err(e);
    if (st != 0) return st;  // BS_EINVAL (a point of an invalid kind) or BS_TIMEOUT
  }
  return BS_OK;
}

int pinn_train_step(pinn_model* m, const double* X, const int8_t* kind, int64_t N, const bs_params* prob_params,
                    double smax_over_K, int prec, double lr, double* loss3, double* grad_out, void* stream) {
  Range range_("pinn_train_step");
  return train_step_common(m, X, kind, nullptr, N, prob_params, smax_over_K, prec, lr, loss3, grad_out, stream);
}

int pinn_train_step_data(pinn_model* m, const double* X, const int8_t* kind, const double* y, int64_t N,
                         const bs_params* prob_params, double smax_over_K, int prec, double lr, double* loss3,
                         double* grad_out, void* stream) {
  Range range_("pinn_train_step_data");
  if (!y) return BS_EINVAL;
  return train_step_common(m, X, kind, y, N, prob_params, smax_over_K, prec, lr, loss3, grad_out, stream);
}

// ---------------------------------------------------------------------------
// Parareal
// ---------------------------------------------------------------------------

static cudaError_t ensure_parareal_ws(bs_problem* prob, int max_iter, int d_in) {
  cudaError_t e = cudaSuccess;
  if (!prob->buf0) {
    if ((e = dalloc(&prob->buf0, prob->total_state)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->buf1, prob->total_state)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->fbuf, prob->total_slice)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->gold, prob->total_slice)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->gtab, prob->total_state)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->normbuf, 2 * prob->total_norm)) != cudaSuccess) return e;
    if ((e = dalloc(&prob->ctrl, prob->n_inst)) != cudaSuccess) return e;
    if ((e = cudaMemset(prob->normbuf, 0, sizeof(double) * 2 * prob->total_norm)) != cudaSuccess) return e;
  }
  if (max_iter > prob->norms_cap) {
    cudaFree(prob->norms_dev);
    prob->norms_dev = nullptr;
    if ((e = dalloc(&prob->norms_dev, (size_t)prob->n_inst * max_iter)) != cudaSuccess) return e;
    prob->norms_cap = max_iter;
  }
  if (d_in > 0 && prob->xgrid_din != d_in) {
    cudaFree(prob->Xgrid);
    prob->Xgrid = nullptr;
    if ((e = dalloc(&prob->Xgrid, (size_t)prob->total_state * d_in)) != cudaSuccess) return e;
    prob->xgrid_din = d_in;
  }
  return e;
}

// Arguments common to both solve entry points (nothing launched on error).
static int solve_args_ok(const bs_problem* prob, int coarse_kind, const pinn_model* model, int prec, double tol,
                         int32_t max_iter, const double* U_out) {
  if (!prob || !U_out || ((uintptr_t)U_out & 15) || max_iter < 1 || !(tol >= 0.0)) return BS_EINVAL;
  if (coarse_kind < BS_COARSE_IE || coarse_kind > BS_COARSE_PINN_IE) return BS_EINVAL;
  const bool pinn = coarse_kind != BS_COARSE_IE;
  if (pinn && !model) return BS_EINVAL;
  if (pinn && (prec < BS_FP64 || prec > BS_BF16)) return BS_EINVAL;
  return BS_OK;
}

// Device workspace of one solve: on the problem handle (parareal_solve) or in
// the fixed array (parareal_solve_static).
struct SolveWs {
  double *buf0, *buf1;  // U^k / U^{k+1} ping-pong (state layout)
  double* fbuf;         // F(U^k_n) (slice layout)
  double* gold;         // G(U^k_n) (slice layout)
  double* gtab;         // network table (state layout)
  double* xg;           // grid points of the table, d_in per point
  double* normbuf;      // increment-norm partial sums
  bsp::Ctrl* ctrl;      // per-instance control words
  double* norms;        // increment-norm history, n_inst x max_iter
  bool clear_normbuf;   // zero the partial sums first (the array keeps the last call's)
};

// One Parareal solve (Eq. 7) of every instance of the problem, enqueued on s:
//   a1 network table, a2 initial iterate, then per iteration a3 fine
//   propagation (+ a5 fused for the state-independent network coarse), a4 + a5
//   the serial coarse sweep with the correction, and the stop test; the stop
//   rule is decided on the device, so the launch sequence is fixed.
// hc: host space for n_inst control words when norms or stats are wanted.
static int solve_impl(bs_problem* prob, int coarse_kind, const pinn_model* model, int prec, double tol,
                      int32_t max_iter, double* U_out, double* norms, bs_instance_stats* stats, cudaStream_t s,
                      const SolveWs& w, bsp::Ctrl* hc) {
  const bool pinn = coarse_kind != BS_COARSE_IE;
  const int n = prob->n_inst;
  cudaError_t e = cudaSuccess;
  if (w.clear_normbuf &&
      (e = cudaMemsetAsync(w.normbuf, 0, sizeof(double) * 2 * prob->total_norm, s)) != cudaSuccess)
    return map_err(e);
  if ((e = cudaMemsetAsync(prob->d_sched, 0, sizeof(int) * (size_t)prob->sched_n, s)) != cudaSuccess)
    return map_err(e);
  const int ncls = (int)prob->classes.size();
  int* live = prob->d_sched + (int64_t)(prob->maxP + 1) * ncls;  // live[k]: after iteration k
  // a1: network table on (S_j, tau_n), Dirichlet nodes exact
  if (pinn) {
    Range r("network table");
    const int d_in = model->dev.d_in;
    if ((e = bsp::launch_grid_points(prob->d_insts, n, d_in, w.xg, s)) != cudaSuccess) return map_err(e);
    if ((e = bsp::launch_mlp_eval(model->dev, prec, w.xg, prob->total_state, w.gtab, nullptr, s)) != cudaSuccess)
      return map_err(e);
    if ((e = bsp::launch_table_fix(prob->d_insts, n, prob->exptab, w.gtab, s)) != cudaSuccess) return map_err(e);
  }
  // network-anchored IE: c_n = g_{n+1} - IE(g_n) for every slice at once (IE
  // over all slices of the table into fbuf, which iteration 0 overwrites)
  if (coarse_kind == BS_COARSE_PINN_IE) {
    for (auto& c : prob->classes) {
      bsp::PropArgs a{};
      a.insts = prob->d_insts;
      a.ids = c.d_ids;
      a.pool = prob->pool;
      a.exptab = prob->exptab;
      a.in = w.gtab;
      a.in_state = 1;
      a.out = w.fbuf;
      a.out_state = 0;
      a.mode = bsp::PropArgs::kPlain;
      a.k_iter = -1;
      a.status = prob->d_status;
      if ((e = bsp::launch_prop(c.M, c.NW, c.C, 1, false, a, (int)c.ids.size(), c.maxP, s)) != cudaSuccess)
        return map_err(e);
    }
    if ((e = bsp::launch_table_correction(prob->d_insts, n, w.fbuf, w.gtab, s)) != cudaSuccess) return map_err(e);
  }
  // a2: initial iterate
  if ((e = bsp::launch_parareal_init(prob->d_insts, n, w.buf0, w.buf1, w.gtab, coarse_kind == BS_COARSE_PINN, w.ctrl,
                                     w.norms, max_iter, s)) != cudaSuccess)
    return map_err(e);
  const int sweep_kind = coarse_kind == BS_COARSE_IE ? 0 : coarse_kind == BS_COARSE_PINN_INCR ? 1 : 2;
  auto sweep = [&](int k, double* cur, double* nxt) -> cudaError_t {
    for (auto& c : prob->classes) {
      bsp::SweepArgs a{};
      a.insts = prob->d_insts;
      a.ids = c.d_ids;
      a.pool = prob->pool;
      a.exptab = prob->exptab;
      a.kind = sweep_kind;
      a.k_iter = k;
      a.ctrl = k < 0 ? nullptr : w.ctrl;
      a.n_live = k > 0 ? live + (k - 1) : nullptr;
      a.ucur = cur;
      a.unext = nxt;
      a.gold = w.gold;
      a.fbuf = w.fbuf;
      a.gtab = w.gtab;
      a.normbuf = w.normbuf;
      a.status = prob->d_status;
      cudaError_t ee = bsp::launch_sweep(c.M, c.NW, c.C, a, (int)c.ids.size(), s);
      if (ee != cudaSuccess) return ee;
    }
    return cudaSuccess;
  };
  if (coarse_kind != BS_COARSE_PINN) {
    if ((e = sweep(-1, w.buf0, w.buf0)) != cudaSuccess) return map_err(e);
  }
  const int kmax = max_iter < prob->maxP ? max_iter : prob->maxP;
  for (int k = 0; k < kmax; ++k) {
    Range r("parareal iteration");
    double* cur = (k & 1) ? w.buf1 : w.buf0;
    double* nxt = (k & 1) ? w.buf0 : w.buf1;
    // a3 (+ a5 fused for the state-independent network coarse propagator)
    for (int ci = 0; ci < ncls; ++ci) {
      const auto& c = prob->classes[ci];
      bsp::PropArgs a{};
      a.task_ctr = prob->d_sched + (int64_t)(k + 1) * ncls + ci;
      a.n_live = k > 0 ? live + (k - 1) : nullptr;
      a.insts = prob->d_insts;
      a.ids = c.d_ids;
      a.pool = prob->pool;
      a.exptab = prob->exptab;
      a.in = cur;
      a.in_state = 1;
      a.k_iter = k;
      a.ctrl = w.ctrl;
      a.status = prob->d_status;
      if (coarse_kind == BS_COARSE_PINN) {
        a.out = nxt;
        a.out_state = 1;
        a.mode = bsp::PropArgs::kPinnFused;
        a.uold = cur;
        a.normbuf = w.normbuf;
      } else {
        a.out = w.fbuf;
        a.out_state = 0;
        a.mode = bsp::PropArgs::kPlain;
      }
      if ((e = bsp::launch_prop(c.M, c.NW, c.C, c.s2, true, a, (int)c.ids.size(), c.maxP, s)) != cudaSuccess)
        return map_err(e);
    }
    // a4 + a5: serial coarse sweep with the correction
    if (coarse_kind != BS_COARSE_PINN) {
      if ((e = sweep(k, cur, nxt)) != cudaSuccess) return map_err(e);
    }
    if ((e = bsp::launch_parareal_finalize(prob->d_insts, n, w.normbuf, k, tol, max_iter, w.ctrl, w.norms, live + k,
                                           s)) != cudaSuccess)
      return map_err(e);
  }
  if ((e = bsp::launch_copy_result(prob->d_insts, n, w.ctrl, w.buf0, w.buf1, U_out, s)) != cudaSuccess)
    return map_err(e);
  if (!norms && !stats) return BS_OK;
  int dev_status = 0;
  if ((e = cudaMemcpyAsync(hc, w.ctrl, sizeof(bsp::Ctrl) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return map_err(e);
  if ((e = cudaMemcpyAsync(&dev_status, prob->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return map_err(e);
  if (norms && (e = cudaMemcpyAsync(norms, w.norms, sizeof(double) * (size_t)n * max_iter, cudaMemcpyDeviceToHost,
                                    s)) != cudaSuccess)
    return map_err(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_err(e);
  int worst = BS_OK;
  for (int i = 0; i < n; ++i) {
    if (stats) {
      stats[i].iterations = hc[i].iterations;
      stats[i].status = hc[i].status;
      stats[i].final_norm = hc[i].last_norm;
    }
    if (hc[i].status != BS_OK && (worst == BS_OK || hc[i].status == BS_DIVERGED)) worst = hc[i].status;
  }
  return dev_status != 0 ? BS_TIMEOUT : worst;
}

int parareal_solve(bs_problem* prob, int coarse_kind, const pinn_model* model, int prec, double tol,
                   int32_t max_iter, double* U_out, double* norms, bs_instance_stats* stats, void* stream) {
  Range range_("parareal_solve");
  const int rc = solve_args_ok(prob, coarse_kind, model, prec, tol, max_iter, U_out);
  if (rc != BS_OK) return rc;
  const bool pinn = coarse_kind != BS_COARSE_IE;
  cudaError_t e = ensure_parareal_ws(prob, max_iter, pinn ? model->dev.d_in : 0);
  if (e != cudaSuccess) return map_err(e);
  SolveWs w{prob->buf0, prob->buf1, prob->fbuf, prob->gold, prob->gtab, prob->Xgrid,
            prob->normbuf, prob->ctrl, prob->norms_dev, false};
  std::vector<bsp::Ctrl> hc(norms || stats ? prob->n_inst : 0);
  return solve_impl(prob, coarse_kind, model, prec, tol, max_iter, U_out, norms, stats, (cudaStream_t)stream, w,
                    hc.data());
}

}  // extern "C"

// ---------------------------------------------------------------------------
// parareal_solve_static: the same solve with its workspace in a fixed device
// array instead of memory allocated on the problem handle.
//
// Who needs it: callers that must not allocate device memory once set-up is
// done -- code that enqueues work while a stream is being captured, loops
// where a cudaMalloc/cudaFree would synchronise the device and stall other
// streams, and processes whose device memory is already reserved by another
// allocator (parareal_solve allocates its workspace on the first call for a
// problem).  This entry point calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array is a file-scope __device__ object of kStaticScratchBytes; every
// GPU that loads this library keeps it until the process exits.  Its name is
// only a host-side stand-in, so host code asks for its device address with
// cudaGetSymbolAddress, once per device, on that device's first call.  That
// first call should therefore come before any stream capture.  All calls share
// the array and it keeps the previous call's contents: the parts that must
// start cleared are cleared by each call, and calls whose work overlaps on the
// GPU (two streams, or two host threads) race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;  // 16 MiB
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticMaxInstances = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

cudaError_t static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int parareal_solve_static(bs_problem* prob, int coarse_kind, const pinn_model* model, int prec,
                                     double tol, int32_t max_iter, double* U_out, double* norms,
                                     bs_instance_stats* stats, void* stream) {
  Range range_("parareal_solve_static");
  const int rc = solve_args_ok(prob, coarse_kind, model, prec, tol, max_iter, U_out);
  if (rc != BS_OK) return rc;
  const bool pinn = coarse_kind != BS_COARSE_IE;
  const int n = prob->n_inst;
  if (n > kStaticMaxInstances) return BS_EUNSUPPORTED;
  const int d_in = pinn ? model->dev.d_in : 0;
  // carve the fixed array: two state buffers, F, G_old, network table, grid
  // points, norm partial sums, control words, norm history
  size_t off = 0;
  const size_t o_buf0 = off;
  off = align256(off + sizeof(double) * prob->total_state);
  const size_t o_buf1 = off;
  off = align256(off + sizeof(double) * prob->total_state);
  const size_t o_fbuf = off;
  off = align256(off + sizeof(double) * prob->total_slice);
  const size_t o_gold = off;
  off = align256(off + sizeof(double) * prob->total_slice);
  const size_t o_gtab = off;
  off = align256(off + sizeof(double) * prob->total_state);
  const size_t o_xg = off;
  off = align256(off + sizeof(double) * prob->total_state * (size_t)d_in);
  const size_t o_nb = off;
  off = align256(off + sizeof(double) * 2 * prob->total_norm);
  const size_t o_ctrl = off;
  off = align256(off + sizeof(bsp::Ctrl) * n);
  const size_t o_norms = off;
  off = align256(off + sizeof(double) * (size_t)n * max_iter);
  if (off > kStaticScratchBytes) return BS_EUNSUPPORTED;  // problem too large for the fixed array
  void* base = nullptr;
  cudaError_t e = static_scratch_address(&base);
  if (e != cudaSuccess) return map_err(e);
  unsigned char* b = static_cast<unsigned char*>(base);
  SolveWs w{reinterpret_cast<double*>(b + o_buf0),  reinterpret_cast<double*>(b + o_buf1),
            reinterpret_cast<double*>(b + o_fbuf),  reinterpret_cast<double*>(b + o_gold),
            reinterpret_cast<double*>(b + o_gtab),  reinterpret_cast<double*>(b + o_xg),
            reinterpret_cast<double*>(b + o_nb),    reinterpret_cast<bsp::Ctrl*>(b + o_ctrl),
            reinterpret_cast<double*>(b + o_norms), true};
  bsp::Ctrl hc[kStaticMaxInstances];  // host control words without a heap allocation
  return solve_impl(prob, coarse_kind, model, prec, tol, max_iter, U_out, norms, stats, (cudaStream_t)stream, w, hc);
}
