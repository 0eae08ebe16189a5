// batch.cu -- batches of uneven birth-death instances (the C ABI's
// expv_batch_*): one R-MJP series per instance, many instances per call.
//
// Scheduling on GB300: every instance is a chain of K_j jumps over N_j
// states, so its work is ~K_j N_j and the work spans several decades.  The
// instances are sorted longest first and launched as one grid per group, so
// the hardware block scheduler hands the longest remaining instance to the
// next free SM (list scheduling, longest processing time first).  Instances
// whose work alone would exceed a fair share of the makespan ("heavy") are
// split over a thread-block cluster, so the largest instance does not set the
// makespan; the light ones run one CTA each, grouped by size so each group
// gets a fitting CTA width.  The groups run concurrently on separate streams;
// the whole sequence can be captured as one CUDA graph.
//
// Two chain kernels serve the groups: the register-resident one
// (stencil_reg1d.cu; clusters exchange halos every h jumps), the default
// wherever every instance fits it, and the shared-memory one (stencil.cu;
// clusters exchange boundary values every jump), which takes any size.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "host_util.h"
#include "internal.cuh"

using namespace mjp;

namespace {

constexpr int kGroups = 16;        // groups of either kernel at most
constexpr int kClassicGroups = 4;  // shared-memory kernel: heavy + three light size classes
constexpr int kMaxRegCluster = 8;  // register kernel: CTAs per instance at most
constexpr size_t kSmemMax = 227 * 1024;

struct Group {
  std::vector<int32_t> jobs;  // longest first
  int cluster = 1, threads = 128, tile = 0;
  size_t smem = 0;
  bool reg = false;  // register-resident kernel (plan in rp)
  Reg1dPlan rp = {};
  DevBuf d_map;
};

// Largest exit rate of a birth-death chain (reflecting top), for the work
// estimate only (the device planner computes the exact Omega).
double bd_max_exit(int64_t N, double b, double g) {
  if (N <= 1) return 0.0;
  double top = g * (double)(N - 1);
  double mid = b + g * (double)(N - 2);
  return std::max(top, mid);
}

}  // namespace

struct mjp_batch {
  int kind = MJP_BD1D, precision = MJP_FP32, n = 0;
  std::vector<int64_t> N, s0, off;
  std::vector<double> theta, t, work;
  // launch configuration (tuned)
  int light_threads[3] = {96, 288, 608};
  int heavy_cluster = 8, heavy_threads = 288;
  double heavy_factor = 1.0;
  // register-resident kernel: 0 = automatic, 1 = shared-memory kernel only,
  // 2 = register kernel only (MJP_OPT_CHAIN)
  int chain = 0;
  int reg_heavy_cluster = 4, reg_halo = 32;
  double reg_heavy_factor = 1.0;
  int renorm = kDefectPeriod;  // FP32: exit-defect correction period (MJP_OPT_RENORM_PERIOD)
  int sms = 152;
  Group groups[kGroups];
  bool uploaded = false, grouped = false;
  DevBuf d_theta, d_times, d_jobN, d_off, d_s0, d_win, d_info, d_comp, d_status;
  DevBuf d_arena, d_arena_ctl;  // planner's Poisson-weight store and its counters
  int64_t arena_cap = 0;
  cudaStream_t side[kGroups] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kGroups] = {};
  cudaGraphExec_t exec = nullptr;
  void* g_out = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (the legacy stream cannot be captured)
  ~mjp_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    for (auto& s : side)
      if (s) cudaStreamDestroy(s);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto& e : ev_join)
      if (e) cudaEventDestroy(e);
    for (auto& g : groups) g.d_map.release();
    d_theta.release(); d_times.release(); d_jobN.release(); d_off.release(); d_s0.release();
    d_win.release(); d_info.release(); d_comp.release(); d_status.release();
    d_arena.release(); d_arena_ctl.release();
  }
};

namespace {

int tile_of(int64_t N, int cluster) {
  int64_t slab = (N + cluster - 1) / cluster;
  return chain_stencil_tile(MJP_BD1D, N, 1, slab);
}

// Shared-memory kernel: the heavy group and three light size classes.
int regroup_classic(mjp_batch* b) {
  double total = 0.0;
  for (double w : b->work) total += w;
  const double fair = total / std::max(1, b->sms);
  for (auto& g : b->groups) {
    g.jobs.clear();
    g.reg = false;
  }
  for (int j = 0; j < b->n; ++j) {
    int C1tile = tile_of(b->N[j], 1);
    size_t smem1 = chain_stencil_smem_tile(b->precision, 0, C1tile, 1, 0, 0);
    bool heavy = b->work[j] > b->heavy_factor * fair || smem1 > kSmemMax;
    int gi = heavy ? 0 : (b->N[j] < 1024 ? 1 : (b->N[j] < 4096 ? 2 : 3));
    b->groups[gi].jobs.push_back(j);
  }
  for (int gi = 0; gi < kClassicGroups; ++gi) {
    Group& g = b->groups[gi];
    std::stable_sort(g.jobs.begin(), g.jobs.end(), [&](int32_t a, int32_t c) { return b->work[a] > b->work[c]; });
    g.cluster = gi == 0 ? b->heavy_cluster : 1;
    g.threads = gi == 0 ? b->heavy_threads : b->light_threads[gi - 1];
    int tile = 0;
    for (int32_t j : g.jobs) tile = std::max(tile, tile_of(b->N[j], g.cluster));
    while (gi == 0 && !g.jobs.empty() && chain_stencil_smem_tile(b->precision, 0, tile, 1, 0, 0) > kSmemMax &&
           g.cluster < 16) {
      g.cluster *= 2;
      tile = 0;
      for (int32_t j : g.jobs) tile = std::max(tile, tile_of(b->N[j], g.cluster));
    }
    g.tile = tile;
    g.smem = chain_stencil_smem_tile(b->precision, 0, tile, 1, 0, 0);
    if (!g.jobs.empty() && g.smem > kSmemMax) return fail(MJP_ERR_UNSUPPORTED, "an instance does not fit on chip");
    if (!g.jobs.empty()) {  // set kernel attributes now (never inside graph capture)
      ChainParams prep = {};
      prep.B = 0;
      prep.tile_max = g.tile;
      prep.ntimes = 1;
      MJP_CUDA(launch_chain_stencil(MJP_BD1D, b->precision, 0, prep, g.cluster, g.threads, nullptr));
    }
    int rc = g.d_map.ensure(sizeof(int32_t) * std::max<size_t>(1, g.jobs.size()));
    if (rc) return rc;
    if (!g.jobs.empty())
      MJP_CUDA(cudaMemcpy(g.d_map.p, g.jobs.data(), sizeof(int32_t) * g.jobs.size(), cudaMemcpyHostToDevice));
  }
  return MJP_OK;
}


// Register kernel: every instance takes the fewest CTAs that hold it (at
// most kMaxRegCluster), heavy ones at least reg_heavy_cluster; one group per
// cluster size, and six size classes of single-CTA instances (a CTA is as wide
// as its group's largest instance needs, so classes keep idle threads few).
// Returns MJP_ERR_UNSUPPORTED when some instance fits no cluster.
int regroup_reg(mjp_batch* b) {
  double total = 0.0;
  for (double w : b->work) total += w;
  const double fair = total / std::max(1, b->sms);
  const int64_t per_cta = chain_reg1d_max_states(b->precision);
  std::vector<int> gof(b->n);
  Reg1dPlan rp;
  for (int j = 0; j < b->n; ++j) {
    int c = 1;
    while (c <= kMaxRegCluster && !chain_reg1d_plan(b->precision, b->N[j], 1, c, b->reg_halo, &rp)) ++c;
    if (c > kMaxRegCluster) return fail(MJP_ERR_UNSUPPORTED, "an instance does not fit the register-resident chain");
    if (b->work[j] > b->reg_heavy_factor * fair)
      for (int ch = std::min(b->reg_heavy_cluster, kMaxRegCluster); ch > c; --ch)
        if (chain_reg1d_plan(b->precision, b->N[j], 1, ch, b->reg_halo, &rp)) {
          c = ch;
          break;
        }
    // groups 0..5: one CTA, up to 1/16, 1/8, 1/4, 1/2, 3/4 and all of a
    // CTA's states; group 4 + c: clusters of c CTAs
    int cls = 5;
    if (c == 1) {
      const int64_t n16 = b->N[j] * 16;
      cls = n16 <= per_cta ? 0 : n16 <= 2 * per_cta ? 1 : n16 <= 4 * per_cta ? 2 : n16 <= 8 * per_cta ? 3
                                                                                 : n16 <= 12 * per_cta ? 4 : 5;
    }
    gof[j] = c > 1 ? 4 + c : cls;
  }
  for (auto& g : b->groups) {
    g.jobs.clear();
    g.reg = true;
  }
  for (int j = 0; j < b->n; ++j) b->groups[gof[j]].jobs.push_back(j);
  for (int gi = 0; gi < kGroups; ++gi) {
    Group& g = b->groups[gi];
    if (g.jobs.empty()) continue;
    std::stable_sort(g.jobs.begin(), g.jobs.end(), [&](int32_t a, int32_t c) { return b->work[a] > b->work[c]; });
    int64_t nmax = 0;
    for (int32_t j : g.jobs) nmax = std::max(nmax, b->N[j]);
    const int C = gi <= 5 ? 1 : gi - 4;
    if (!chain_reg1d_plan(b->precision, nmax, 1, C, b->reg_halo, &g.rp))
      return fail(MJP_ERR_UNSUPPORTED, "a batch group does not fit the register-resident chain");
    g.cluster = C;
    g.threads = g.rp.threads;
    g.smem = g.rp.smem;
    ChainParams prep = {};  // set kernel attributes now (never inside graph capture)
    prep.B = 0;
    MJP_CUDA(launch_chain_reg1d(b->precision, prep, g.rp, nullptr));
    int rc = g.d_map.ensure(sizeof(int32_t) * g.jobs.size());
    if (rc) return rc;
    MJP_CUDA(cudaMemcpy(g.d_map.p, g.jobs.data(), sizeof(int32_t) * g.jobs.size(), cudaMemcpyHostToDevice));
  }
  return MJP_OK;
}

int regroup(mjp_batch* b) {
  int rc = MJP_ERR_UNSUPPORTED;
  if (b->chain != 1) rc = regroup_reg(b);
  if (rc && b->chain != 2) rc = regroup_classic(b);
  if (rc) return rc;
  b->grouped = true;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return MJP_OK;
}

int upload(mjp_batch* b) {
  const int n = b->n;
  const size_t elt = b->precision == MJP_FP64 ? 8 : 4;
  int rc = 0;
  if ((rc = b->d_theta.ensure(sizeof(double) * 2 * n)) || (rc = b->d_times.ensure(sizeof(double) * n)) ||
      (rc = b->d_jobN.ensure(sizeof(int32_t) * n)) || (rc = b->d_off.ensure(sizeof(int64_t) * n)) ||
      (rc = b->d_s0.ensure(sizeof(int64_t) * n)) || (rc = b->d_win.ensure(sizeof(Win) * n)) ||
      (rc = b->d_info.ensure(sizeof(JobInfo) * n)) || (rc = b->d_status.ensure(sizeof(int))))
    return rc;
  if (b->precision == MJP_FP32 && (rc = b->d_comp.ensure(sizeof(float) * b->off[n]))) return rc;
  // Every window holds at most 16 sqrt(x) + 3 weights, x = Omega t (Omega is
  // known exactly here: the birth-death maximum exit rate).
  double need = 0.0;
  for (int j = 0; j < n; ++j) need += 16.0 * std::sqrt(1.1 * bd_max_exit(b->N[j], b->theta[2 * j], b->theta[2 * j + 1]) * b->t[j]) + 4.0;
  b->arena_cap = (int64_t)std::min(need, 2.0e9);
  if ((rc = b->d_arena.ensure(elt * (size_t)b->arena_cap)) || (rc = b->d_arena_ctl.ensure(16))) return rc;
  std::vector<int32_t> n32(b->N.begin(), b->N.end());
  MJP_CUDA(cudaMemcpy(b->d_theta.p, b->theta.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice));
  MJP_CUDA(cudaMemcpy(b->d_times.p, b->t.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  MJP_CUDA(cudaMemcpy(b->d_jobN.p, n32.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  MJP_CUDA(cudaMemcpy(b->d_off.p, b->off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  MJP_CUDA(cudaMemcpy(b->d_s0.p, b->s0.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  MJP_CUDA(cudaMemset(b->d_status.p, 0, sizeof(int)));
  for (int gi = 0; gi < kGroups; ++gi) {
    if (!b->side[gi]) MJP_CUDA(cudaStreamCreateWithFlags(&b->side[gi], cudaStreamNonBlocking));
    if (!b->ev_join[gi]) MJP_CUDA(cudaEventCreateWithFlags(&b->ev_join[gi], cudaEventDisableTiming));
  }
  if (!b->ev_fork) MJP_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  b->uploaded = true;
  return MJP_OK;
}

// The launch sequence: planner on `s`, then every non-empty group on its own
// stream, joined back into `s`.
int enqueue(mjp_batch* b, void* out, cudaStream_t s) {
  PlanParams pp = {};
  pp.kind = MJP_BD1D; pp.M = 1; pp.P = 1; pp.N = 1; pp.ntheta = 2; pp.theta = b->d_theta.as<double>();
  pp.B = b->n; pp.ntimes = 1; pp.times = b->d_times.as<double>(); pp.times_per_job = 1;
  pp.trunc_mode = MJP_TRUNC_PAPER; pp.tol = 0.0; pp.omega_factor = 1.1; pp.omega_fixed = -1.0;
  pp.kcap = (int64_t)1 << 26; pp.win = b->d_win.as<Win>(); pp.info = b->d_info.as<JobInfo>();
  pp.status = b->d_status.as<int>(); pp.jobN = b->d_jobN.as<int32_t>();
  pp.arena = b->d_arena.p; pp.arena_cap = b->arena_cap;
  pp.arena_used = b->d_arena_ctl.as<unsigned long long>();
  pp.arena_over = reinterpret_cast<int*>(b->d_arena_ctl.as<char>() + 8);
  pp.arena_fp64 = b->precision == MJP_FP64 ? 1 : 0;
  pp.fp64_weights = pp.arena_fp64;
  MJP_CUDA(cudaMemsetAsync(b->d_arena_ctl.p, 0, 16, s));
  MJP_CUDA(launch_plan(pp, s));
  MJP_CUDA(cudaEventRecord(b->ev_fork, s));
  for (int gi = 0; gi < kGroups; ++gi) {
    Group& g = b->groups[gi];
    if (g.jobs.empty()) continue;
    MJP_CUDA(cudaStreamWaitEvent(b->side[gi], b->ev_fork, 0));
    ChainParams cp = {};
    cp.M = 1; cp.P = 1; cp.N = 1; cp.ntheta = 2; cp.theta = pp.theta; cp.B = (int)g.jobs.size();
    cp.ntimes = 1; cp.orig = nullptr; cp.win = pp.win; cp.info = pp.info; cp.rho0 = nullptr;
    cp.out = out; cp.out_stride = 0; cp.comp = b->d_comp.as<float>(); cp.comp_stride = 0;
    cp.renorm = b->precision == MJP_FP32 ? b->renorm : 0; cp.slab = 1; cp.status = pp.status;
    cp.jobN = pp.jobN; cp.job_off = b->d_off.as<int64_t>(); cp.job_map = g.d_map.as<int32_t>();
    cp.job_s0 = b->d_s0.as<int64_t>(); cp.tile_max = g.tile; cp.arena = b->d_arena.p;
    if (g.reg) MJP_CUDA(launch_chain_reg1d(b->precision, cp, g.rp, b->side[gi]));
    else MJP_CUDA(launch_chain_stencil(MJP_BD1D, b->precision, 0, cp, g.cluster, g.threads, b->side[gi]));
    MJP_CUDA(cudaEventRecord(b->ev_join[gi], b->side[gi]));
    MJP_CUDA(cudaStreamWaitEvent(s, b->ev_join[gi], 0));
  }
  return MJP_OK;
}

int prepare(mjp_batch* b) {
  int rc = 0;
  if (!b->uploaded && (rc = upload(b))) return rc;
  if (!b->grouped && (rc = regroup(b))) return rc;
  return MJP_OK;
}

}  // namespace

extern "C" {

int expv_batch_create(mjp_batch** out, int kind, int n_inst, const int64_t* N, const double* theta,
                      const double* t, const int64_t* s0, int precision) try {
  if (!out) return fail(MJP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (kind != MJP_BD1D) return fail(MJP_ERR_UNSUPPORTED, "batches hold birth-death instances (MJP_BD1D)");
  if (n_inst < 1 || !N || !theta || !t) return fail(MJP_ERR_ARG, "empty batch or NULL array");
  if (precision != MJP_FP32 && precision != MJP_FP64) return fail(MJP_ERR_ARG, "precision must be MJP_FP32 or MJP_FP64");
  auto* b = new mjp_batch();
  b->kind = kind;
  b->precision = precision;
  b->n = n_inst;
  b->N.assign(N, N + n_inst);
  b->theta.assign(theta, theta + 2 * (size_t)n_inst);
  b->t.assign(t, t + n_inst);
  b->s0.assign(n_inst, 0);
  b->off.assign(n_inst + 1, 0);
  b->work.assign(n_inst, 0.0);
  for (int j = 0; j < n_inst; ++j) {
    if (N[j] < 1 || N[j] > 1000000) { delete b; return fail(MJP_ERR_ARG, "instance size must be in [1, 1e6]"); }
    for (int q = 0; q < 2; ++q)
      if (!(theta[2 * j + q] >= 0.0) || !std::isfinite(theta[2 * j + q])) {
        delete b;
        return fail(MJP_ERR_ARG, "rates must be finite and >= 0");
      }
    if (!(t[j] >= 0.0) || !std::isfinite(t[j])) { delete b; return fail(MJP_ERR_ARG, "times must be finite and >= 0"); }
    if (s0) {
      if (s0[j] < 0 || s0[j] >= N[j]) { delete b; return fail(MJP_ERR_ARG, "s0 out of range"); }
      b->s0[j] = s0[j];
    }
    b->off[j + 1] = b->off[j] + N[j];
    double x = 1.1 * bd_max_exit(N[j], theta[2 * j], theta[2 * j + 1]) * t[j];
    double K = std::floor(x + 6.0 * std::sqrt(x)) + 1.0;
    b->work[j] = K * (double)N[j];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) b->sms = v;
  }
  cudaGetLastError();
  *out = b;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int expv_batch_offsets(const mjp_batch* b, int64_t* offsets) try {
  if (!b || !offsets) return fail(MJP_ERR_ARG, "NULL argument");
  std::copy(b->off.begin(), b->off.end(), offsets);
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int expv_batch_run(mjp_batch* b, void* out, int use_graph, void* stream) try {
  if (!b || !out) return fail(MJP_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare(b);
  if (rc) return rc;
  if (!use_graph) return enqueue(b, out, s);
  if (!b->exec || b->g_out != out) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (!b->cap) MJP_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    MJP_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    rc = enqueue(b, out, b->cap);
    cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce != cudaSuccess) return fail(MJP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      b->exec = nullptr;
      return fail(MJP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    }
    b->g_out = out;
  }
  MJP_CUDA(cudaGraphLaunch(b->exec, s));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int expv_batch_check(mjp_batch* b, void* stream) try {
  if (!b) return fail(MJP_ERR_ARG, "NULL batch");
  MJP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (!b->d_status.p) return MJP_OK;
  int st = 0;
  MJP_CUDA(cudaMemcpy(&st, b->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
  MJP_CUDA(cudaMemset(b->d_status.p, 0, sizeof(int)));
  if (st == kStatusKcap) return fail(MJP_ERR_KCAP, "truncation index K above the cap");
  if (st) return fail(MJP_ERR_NUMERIC, "device reported a numerical error");
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int expv_batch_tune(mjp_batch* b, void* out, void* stream, char* cfg, int cfg_len) try {
  if (!b || !out) return fail(MJP_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare(b);
  if (rc) return rc;
  struct Cand {
    int chain;  // 1 shared-memory kernel, 2 register kernel
    int lt[3];
    int hc, ht;
    double hf;
  };
  const int user_chain = b->chain;
  std::vector<Cand> cands;
  if (user_chain != 1) {
    b->chain = 2;
    if (regroup(b) == MJP_OK)
      for (int hc : {2, 4, 8})
        for (double hf : {0.5, 1.0, 2.0}) cands.push_back({2, {0, 0, 0}, hc, 0, hf});
  }
  if (user_chain == 1 || (user_chain == 0 && cands.empty())) {
    const int lts[2][3] = {{96, 288, 608}, {64, 160, 416}};
    for (auto& lt : lts)
      for (int hc : {4, 8, 16})
        for (double hf : {0.5, 1.0, 2.0}) cands.push_back({1, {lt[0], lt[1], lt[2]}, hc, hc >= 8 ? 160 : 288, hf});
  } else if (user_chain == 0) {
    cands.push_back({1, {96, 288, 608}, 4, 288, 0.5});  // the shared-memory kernel's usual best, for comparison
  }
  if (cands.empty()) {
    b->chain = user_chain;
    return fail(MJP_ERR_UNSUPPORTED, "no launch configuration fits this batch");
  }
  auto apply = [&](const Cand& c) {
    b->chain = c.chain;
    if (c.chain == 2) {
      b->reg_heavy_cluster = c.hc;
      b->reg_heavy_factor = c.hf;
    } else {
      std::copy(c.lt, c.lt + 3, b->light_threads);
      b->heavy_cluster = c.hc;
      b->heavy_threads = c.ht;
      b->heavy_factor = c.hf;
    }
  };
  cudaEvent_t e0, e1;
  MJP_CUDA(cudaEventCreate(&e0));
  MJP_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  Cand bestc = cands[0];
  rc = MJP_OK;
  for (const Cand& c : cands) {
    apply(c);
    if (regroup(b) != MJP_OK) continue;
    cudaEventRecord(e0, s);
    if (enqueue(b, out, s) != MJP_OK) {  // shape not launchable here: skip it
      cudaStreamSynchronize(s);
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = fail(MJP_ERR_CUDA, "tuning run failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply(bestc);
  int rc2 = regroup(b);
  b->chain = user_chain == 0 ? bestc.chain : user_chain;
  if (rc) return rc;
  if (rc2) return rc2;
  size_t heavy = 0;
  for (int gi = 0; gi < kGroups; ++gi)
    if (b->groups[gi].cluster > 1) heavy += b->groups[gi].jobs.size();
  if (cfg && cfg_len > 0) {
    if (bestc.chain == 2)
      snprintf(cfg, (size_t)cfg_len,
               "{\"chain\": \"register\", \"heavy_cluster\": %d, \"heavy_factor\": %.2f, \"halo\": %d, "
               "\"ms\": %.4f, \"cluster_jobs\": %zu}",
               b->reg_heavy_cluster, b->reg_heavy_factor, b->reg_halo, best, heavy);
    else
      snprintf(cfg, (size_t)cfg_len,
               "{\"chain\": \"shared\", \"light_threads\": [%d, %d, %d], \"heavy_cluster\": %d, "
               "\"heavy_threads\": %d, \"heavy_factor\": %.2f, \"ms\": %.4f, \"cluster_jobs\": %zu}",
               b->light_threads[0], b->light_threads[1], b->light_threads[2], b->heavy_cluster, b->heavy_threads,
               b->heavy_factor, best, heavy);
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int expv_batch_set_option(mjp_batch* b, int option, int64_t value) try {
  if (!b) return fail(MJP_ERR_ARG, "NULL batch");
  switch (option) {
    case MJP_OPT_CHAIN:
      if (value < 0 || value > 2) return fail(MJP_ERR_ARG, "chain must be 0, 1 or 2");
      b->chain = (int)value;
      break;
    case MJP_OPT_CLUSTER:
      if (value < 0 || value > kMaxRegCluster) return fail(MJP_ERR_ARG, "cluster must be in [0, 8]");
      b->reg_heavy_cluster = value == 0 ? 4 : (int)value;
      b->heavy_cluster = value == 0 ? 8 : std::max(2, (int)value);
      break;
    case MJP_OPT_HALO:
      if (value < 1 || value > 1024) return fail(MJP_ERR_ARG, "halo must be in [1, 1024]");
      b->reg_halo = (int)value;
      break;
    case MJP_OPT_RENORM_PERIOD:
      if (value < 0 || value > (1 << 20) || value % 8 != 0)
        return fail(MJP_ERR_ARG, "renorm period must be 0 or a multiple of 8 in [8, 2^20]");
      b->renorm = (int)value;
      break;
    default:
      return fail(MJP_ERR_ARG, "option not supported by batches");
  }
  b->grouped = false;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

void expv_batch_destroy(mjp_batch* b) { delete b; }

}  // extern "C"
