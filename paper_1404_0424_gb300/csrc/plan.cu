// Batched uneven problems: plans, bins, CUDA-graph capture and the schedule
// autotuner behind cg_plan_create / cg_plan_run.
//
// A plan groups its problems into bins by operation, padded user count and
// tracker; each bin runs one persistent warp-per-instance kernel whose warps
// claim (problem, instance) units from a device counter. A schedule fixes
// how: the order in which units are claimed (as given, or longest first, so
// that the long units start early and the short ones fill the tail), whether
// the bins run side by side on forked streams or one after another, what
// share of its resident CTAs each bin's grid takes, and (with CG_PREC_AUTO)
// the split precision. The autotuner times the candidates on the batch
// itself and keeps the fastest per device and shape class (tune.cu).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "cgmimo.h"
#include "host_checks.h"
#include "launch.cuh"
#include "tune.h"

using namespace cgm;

namespace {

struct Bin {
  int op = 0, UT = 0;
  bool full = false;
  int PB = 0, PR = 0, PEX = 0;
  std::vector<int2> work;   // (descriptor, instance), in descriptor order
  std::vector<float> cost;  // estimated cost of each unit (work_cost)
  int64_t work_off = 0;     // offset of this bin's units in the device work array
  int full_grid = 0;        // resident CTAs, at most one per four units
  int grid = 0;             // grid of the schedule in use
};

// Estimated cost of one work unit, in units of tensor-core work: the Gram
// and matched filter over B antennas, K products A p on 16 right-hand-side
// rows (times the exact tracker's recursion), and for precoding q = H v.
float work_cost(const cg_desc& d, int UT) {
  const float B = float(d.B), U = float(UT), R = float(d.R), K = float(d.K);
  if (d.op == CG_OP_DETECT) {
    const float exact = d.sinr_mode == CG_SINR_EXACT ? 1.f + R * U / 8.f : 1.f;
    return B * U * (U / 2.f + R) + K * 16.f * U * U * exact;
  }
  return B * U * U / 2.f + K * 16.f * U * U + B * 16.f * U;
}

int precision_el(int32_t prec) { return (prec == CG_PREC_BF16 || prec == CG_PREC_BF16X3) ? 0 : 1; }
bool precision_x3(int32_t prec) { return prec == CG_PREC_BF16X3 || prec == CG_PREC_FP16X3; }

int check_desc(const cg_desc& d) {
  cg_params p{};
  p.B = d.B;
  p.U = d.U;
  p.qam_bits = d.qam_bits;
  p.K = d.K;
  p.R = d.R;
  p.N0 = d.N0;
  p.Es = d.Es;
  p.sinr_mode = d.sinr_mode;
  p.amul_mode = CG_AMUL_EXPLICIT;
  p.precision = CG_PREC_FP16X3;
  if (d.n_inst < 0) return CG_EINVAL;
  if (d.op == CG_OP_DETECT)
    return check_detect(&p, d.n_inst, d.H, d.in, d.out, d.mu, d.rho, d.aux, d.status);
  if (d.op == CG_OP_PRECODE) return check_precode(&p, d.n_inst, d.H, d.in, d.out, d.aux, d.status);
  return CG_EINVAL;
}

// The autotuner's cache key: device name, then per bin its shape and the
// power of two above its unit count.
std::string shape_key(const std::vector<Bin>& bins, int dev) {
  char name[256] = {0};
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    std::snprintf(name, sizeof(name), "%s", prop.name);
  std::string k = name;
  char buf[96];
  for (const Bin& b : bins) {
    const size_t units = b.work.size();
    int scale = 0;
    while ((size_t(1) << scale) < units) ++scale;
    std::snprintf(buf, sizeof(buf), "|%d,%d,%d,%d,%d,%d,%d", b.op, b.UT, int(b.full), b.PB, b.PR,
                  b.PEX, scale);
    k += buf;
  }
  return k;
}

// Schedule of a plan that asks for a fixed precision: longest first, bins
// side by side, full grids.
TuneEntry default_schedule(int32_t precision) { return TuneEntry{precision, 1, 1, 100, 0.f}; }

}  // namespace

struct cg_plan {
  int dev = 0;
  TuneEntry sched{CG_PREC_FP16X3, 1, 1, 100, 0.f};
  int32_t source = CG_TUNE_FIXED;
  std::vector<Bin> bins;
  void* dmem = nullptr;
  cg_desc* d_desc = nullptr;
  int2* d_work = nullptr;
  unsigned long long* d_counter = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;  // [0] fork, [1..] joins
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int2> staging;    // host copy of the ordered work units
};

namespace {

void release_graph(cg_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

// Uploads every bin's work units in the order of `s` and sets the bins'
// grids; waits for the copy (the host staging is reused).
int apply_order_and_grid(cg_plan* p, const TuneEntry& s) {
  size_t units = 0;
  for (const Bin& b : p->bins) units += b.work.size();
  p->staging.resize(std::max<size_t>(units, 1));
  for (Bin& b : p->bins) {
    std::vector<size_t> idx(b.work.size());
    std::iota(idx.begin(), idx.end(), size_t(0));
    if (s.order == 1)
      std::stable_sort(idx.begin(), idx.end(),
                       [&](size_t x, size_t y) { return b.cost[x] > b.cost[y]; });
    for (size_t i = 0; i < idx.size(); ++i) p->staging[size_t(b.work_off) + i] = b.work[idx[i]];
    b.grid = std::max(1, int((int64_t(b.full_grid) * s.grid_pct + 99) / 100));
  }
  if (units == 0) return CG_OK;
  if (cudaMemcpyAsync(p->d_work, p->staging.data(), sizeof(int2) * units, cudaMemcpyHostToDevice,
                      p->capture) != cudaSuccess ||
      cudaStreamSynchronize(p->capture) != cudaSuccess)
    return CG_ECUDA;
  return CG_OK;
}

// Captures memset(counters) + one persistent kernel per bin into p->graph /
// p->exec: with s.concurrent the bins are forked onto side streams and run
// side by side, otherwise one after another on the capture stream.
int capture(cg_plan* p, const TuneEntry& s) {
  release_graph(p);
  const int el = precision_el(s.precision);
  const bool x3 = precision_x3(s.precision);
  cudaStream_t cs = p->capture;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CG_ECUDA;
  cudaError_t err =
      cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long) * p->bins.size(), cs);
  if (err == cudaSuccess && s.concurrent) err = cudaEventRecord(p->ev[0], cs);
  for (size_t i = 0; i < p->bins.size() && err == cudaSuccess; ++i) {
    const Bin& b = p->bins[i];
    const bool fork = s.concurrent && i > 0;
    cudaStream_t bs = fork ? p->side[i - 1] : cs;
    if (fork) err = cudaStreamWaitEvent(bs, p->ev[0], 0);
    if (err != cudaSuccess) break;
    BatchArgs a{};
    a.desc = p->d_desc;
    a.work = p->d_work + b.work_off;
    a.n_work = int64_t(b.work.size());
    a.counter = p->d_counter + i;
    a.PB = b.PB;
    a.PR = b.PR;
    a.PEX = b.PEX;
    err = launch_batch_tc(b.op, b.UT, el, x3, b.full, a, b.grid, bs, true, nullptr, nullptr);
    if (err == cudaSuccess && fork) {
      err = cudaEventRecord(p->ev[i], bs);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(cs, p->ev[i], 0);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(cs, &g);
  if (err != cudaSuccess || end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  p->graph = g;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
    release_graph(p);
    return CG_ECUDA;
  }
  p->sched = s;
  return CG_OK;
}

int use_schedule(cg_plan* p, const TuneEntry& s) {
  const int rc = apply_order_and_grid(p, s);
  return rc != CG_OK ? rc : capture(p, s);
}

// Mean time of `reps` graph launches after one warm-up (milliseconds).
float time_graph(cg_plan* p, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaGraphLaunch(p->exec, p->capture);
  cudaEventRecord(a, p->capture);
  for (int i = 0; i < reps; ++i) cudaGraphLaunch(p->exec, p->capture);
  cudaEventRecord(b, p->capture);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

// The autotuner: every schedule candidate at FP16X3 (claim order x
// concurrency x grid share), then BF16X3 at the best of them, which it
// replaces only when it is at least 3% faster (FP16X3 keeps 22 significant
// bits to BF16X3's 16). These runs write the plan's outputs.
int autotune(cg_plan* p, TuneEntry* best) {
  std::vector<TuneEntry> cands;
  for (int order : {1, 0}) {
    cands.push_back(TuneEntry{CG_PREC_FP16X3, order, 1, 100, 0.f});
    if (p->bins.size() > 1) {
      cands.push_back(TuneEntry{CG_PREC_FP16X3, order, 1, 50, 0.f});
      cands.push_back(TuneEntry{CG_PREC_FP16X3, order, 0, 100, 0.f});
    }
  }
  bool any = false;
  for (TuneEntry c : cands) {
    if (use_schedule(p, c) != CG_OK) continue;
    c.ms = time_graph(p, 3);
    if (!any || c.ms < best->ms) *best = c;
    any = true;
  }
  if (!any) return CG_ECUDA;
  TuneEntry bf = *best;
  bf.precision = CG_PREC_BF16X3;
  if (use_schedule(p, bf) == CG_OK) {
    bf.ms = time_graph(p, 3);
    if (bf.ms < 0.97f * best->ms) *best = bf;
  }
  return CG_OK;
}

void destroy_plan(cg_plan* p) {
  if (p == nullptr) return;
  if (p->capture) cudaStreamSynchronize(p->capture);
  release_graph(p);
  for (cudaStream_t s : p->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  if (p->capture) cudaStreamDestroy(p->capture);
  if (p->dmem) cudaFree(p->dmem);
  delete p;
}

}  // namespace

extern "C" {

int cg_plan_create(const cg_desc* descs, int64_t n, int32_t precision, void* stream,
                   cg_plan** plan, int64_t* bad_index) {
  if (bad_index) *bad_index = -1;
  if (plan == nullptr || n < 0 || (n > 0 && descs == nullptr)) return CG_EINVAL;
  *plan = nullptr;
  if (precision != CG_PREC_AUTO &&
      (precision < CG_PREC_FP32 || precision > CG_PREC_FP16X3))
    return CG_EINVAL;
  if (precision == CG_PREC_FP32) return CG_ENOTSUP;  // plans run the tensor-core kernels
  for (int64_t i = 0; i < n; ++i) {
    const int rc = check_desc(descs[i]);
    if (rc != CG_OK) {
      if (bad_index) *bad_index = i;
      return rc;
    }
  }
  cg_plan* p = new cg_plan();
  if (cudaGetDevice(&p->dev) != cudaSuccess) {
    delete p;
    return CG_ECUDA;
  }
  // bins by (operation, padded users, FULL, exact tracker); each keeps its
  // largest B and R. Exact-tracker detection has bins of its own so that
  // the other problems keep the approximate tracker's kernels.
  std::map<std::tuple<int, int, int, int>, size_t> index;
  for (int64_t i = 0; i < n; ++i) {
    const cg_desc& d = descs[i];
    if (d.n_inst == 0) continue;
    const int UT = std::max(8, padded_users(d.U));
    const bool full = d.U == UT && d.B % 8 == 0;
    const int exact = (d.op == CG_OP_DETECT && d.sinr_mode == CG_SINR_EXACT) ? 1 : 0;
    const auto key = std::make_tuple(d.op, UT, int(full), exact);
    auto it = index.find(key);
    if (it == index.end()) {
      index[key] = p->bins.size();
      Bin b;
      b.op = d.op;
      b.UT = UT;
      b.full = full;
      p->bins.push_back(b);
      it = index.find(key);
    }
    Bin& b = p->bins[it->second];
    b.PB = std::max(b.PB, d.B);
    b.PR = std::max(b.PR, d.R);
    b.PEX |= exact;
    const float c = work_cost(d, UT);
    for (int64_t k = 0; k < d.n_inst; ++k) {
      b.work.push_back(make_int2(int(i), int(k)));
      b.cost.push_back(c);
    }
  }
  size_t units = 0;
  for (Bin& b : p->bins) {
    b.work_off = int64_t(units);
    units += b.work.size();
  }
  // device copy: descriptors, work units, one counter per bin
  const size_t bytes_desc = sizeof(cg_desc) * size_t(std::max<int64_t>(n, 1));
  const size_t off_work = (bytes_desc + 255) & ~size_t(255);
  const size_t off_cnt = (off_work + sizeof(int2) * std::max<size_t>(units, 1) + 255) & ~size_t(255);
  const size_t total = off_cnt + sizeof(unsigned long long) * std::max<size_t>(p->bins.size(), 1);
  int rc = CG_OK;
  if (cudaMalloc(&p->dmem, total) != cudaSuccess) {
    p->dmem = nullptr;
    destroy_plan(p);
    return CG_ENOMEM;
  }
  p->d_desc = reinterpret_cast<cg_desc*>(p->dmem);
  p->d_work = reinterpret_cast<int2*>(static_cast<char*>(p->dmem) + off_work);
  p->d_counter = reinterpret_cast<unsigned long long*>(static_cast<char*>(p->dmem) + off_cnt);
  if (cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking) != cudaSuccess) rc = CG_ECUDA;
  for (size_t i = 1; i < p->bins.size() && rc == CG_OK; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = CG_ECUDA;
    else p->side.push_back(s);
  }
  for (size_t i = 0; i < std::max<size_t>(p->bins.size(), 1) && rc == CG_OK; ++i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = CG_ECUDA;
    else p->ev.push_back(e);
  }
  if (rc == CG_OK && n > 0) {
    // order after the caller's stream, upload the descriptors and wait (the
    // host array may be reused once the call returns)
    cudaEvent_t ready;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) rc = CG_ECUDA;
    if (rc == CG_OK) {
      if (cudaEventRecord(ready, static_cast<cudaStream_t>(stream)) != cudaSuccess ||
          cudaStreamWaitEvent(p->capture, ready, 0) != cudaSuccess ||
          cudaMemcpyAsync(p->d_desc, descs, sizeof(cg_desc) * size_t(n), cudaMemcpyHostToDevice,
                          p->capture) != cudaSuccess ||
          cudaStreamSynchronize(p->capture) != cudaSuccess)
        rc = CG_ECUDA;
      cudaEventDestroy(ready);
    }
  }
  // full grids: resident CTAs of the bin's kernel, at most one per four units
  for (Bin& b : p->bins) {
    if (rc != CG_OK) break;
    BatchArgs a{};
    a.n_work = int64_t(b.work.size());
    a.PB = b.PB;
    a.PR = b.PR;
    a.PEX = b.PEX;
    const int32_t prec = precision == CG_PREC_AUTO ? CG_PREC_FP16X3 : precision;
    const cudaError_t err = launch_batch_tc(b.op, b.UT, precision_el(prec), precision_x3(prec),
                                            b.full, a, 0, nullptr, false, nullptr, &b.full_grid);
    if (err != cudaSuccess) rc = err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  if (rc == CG_OK && !p->bins.empty()) {
    if (precision != CG_PREC_AUTO) {
      p->source = CG_TUNE_FIXED;
      rc = use_schedule(p, default_schedule(precision));
    } else {
      const std::string key = shape_key(p->bins, p->dev);
      TuneEntry s{};
      if (tune_lookup(key, &s)) {
        p->source = CG_TUNE_CACHED;
        rc = use_schedule(p, s);
      } else {
        rc = autotune(p, &s);
        if (rc == CG_OK) {
          tune_store(key, s);
          p->source = CG_TUNE_TIMED;
          rc = use_schedule(p, s);
        }
      }
    }
  }
  if (rc != CG_OK) {
    destroy_plan(p);
    return rc;
  }
  *plan = p;
  return CG_OK;
}

int cg_plan_run(cg_plan* p, void* stream) {
  if (p == nullptr) return CG_EINVAL;
  if (p->bins.empty()) return CG_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->dev) return CG_EINVAL;
  return cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? CG_OK
                                                                                       : CG_ECUDA;
}

int cg_plan_info(const cg_plan* p, int32_t* precision, int32_t* n_bins) {
  if (p == nullptr) return CG_EINVAL;
  if (precision) *precision = p->sched.precision;
  if (n_bins) *n_bins = int32_t(p->bins.size());
  return CG_OK;
}

int cg_plan_schedule(const cg_plan* p, cg_schedule* out) {
  if (p == nullptr || out == nullptr) return CG_EINVAL;
  out->precision = p->sched.precision;
  out->order = p->sched.order;
  out->concurrent = p->sched.concurrent;
  out->grid_pct = p->sched.grid_pct;
  out->source = p->source;
  out->ms = p->sched.ms;
  return CG_OK;
}

int cg_plan_destroy(cg_plan* p) {
  if (p == nullptr) return CG_EINVAL;
  destroy_plan(p);
  return CG_OK;
}

}  // extern "C"
