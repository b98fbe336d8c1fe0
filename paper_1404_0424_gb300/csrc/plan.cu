// Batched uneven problems: plans, bins, CUDA-graph capture and the precision
// autotuner behind cg_plan_create / cg_plan_run.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cgmimo.h"
#include "host_checks.h"
#include "launch.cuh"

using namespace cgm;

namespace {

struct Bin {
  int op = 0, UT = 0;
  bool full = false;
  int PB = 0, PR = 0, PEX = 0;
  std::vector<int2> work;  // (descriptor, instance)
  int64_t work_off = 0;    // offset of this bin's units in the device work array
  int grid = 0;
};

struct Tuned {
  int32_t precision;
};

std::mutex g_tune_mu;
std::map<std::string, Tuned> g_tune;  // (device, shape class) -> choice

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

// A short description of the plan's shape class, the autotuner's cache key.
std::string shape_key(const std::vector<Bin>& bins, int dev) {
  char name[256] = {0};
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) std::snprintf(name, sizeof(name), "%s", prop.name);
  std::string k = name;
  for (const Bin& b : bins) {
    char buf[96];
    const size_t units = b.work.size();
    int scale = 0;
    while ((size_t(1) << scale) < units) ++scale;  // size class, powers of two
    std::snprintf(buf, sizeof(buf), "|%d,%d,%d,%d,%d,%d,%d", b.op, b.UT, int(b.full), b.PB, b.PR,
                  b.PEX, scale);
    k += buf;
  }
  return k;
}

}  // namespace

struct cg_plan {
  int dev = 0;
  int32_t precision = CG_PREC_FP16X3;
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
};

namespace {

void release_graph(cg_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

// Captures memset(counters) + one persistent kernel per bin (bins forked onto
// side streams so they run concurrently) into p->graph / p->exec.
int capture(cg_plan* p, int32_t precision) {
  release_graph(p);
  const int el = precision_el(precision);
  const bool x3 = precision_x3(precision);
  cudaStream_t s = p->capture;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CG_ECUDA;
  cudaError_t err = cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long) * p->bins.size(), s);
  if (err == cudaSuccess) err = cudaEventRecord(p->ev[0], s);
  for (size_t i = 0; i < p->bins.size() && err == cudaSuccess; ++i) {
    const Bin& b = p->bins[i];
    cudaStream_t bs = i == 0 ? s : p->side[i - 1];
    if (i > 0) err = cudaStreamWaitEvent(bs, p->ev[0], 0);
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
    if (err == cudaSuccess && i > 0) {
      err = cudaEventRecord(p->ev[i], bs);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(s, p->ev[i], 0);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(s, &g);
  if (err != cudaSuccess || end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  p->graph = g;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
    release_graph(p);
    return CG_ECUDA;
  }
  p->precision = precision;
  return CG_OK;
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
  // the other problems keep the warp-per-instance kernels.
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
    if (d.op == CG_OP_DETECT && d.sinr_mode == CG_SINR_EXACT) b.PEX = 1;
    for (int64_t k = 0; k < d.n_inst; ++k) b.work.push_back(make_int2(int(i), int(k)));
  }
  // device copy: descriptors, work units, one counter per bin
  size_t units = 0;
  for (Bin& b : p->bins) {
    b.work_off = int64_t(units);
    units += b.work.size();
  }
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
    // order after the caller's stream, upload, and wait (host vectors are temporary)
    cudaEvent_t ready;
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventRecord(ready, static_cast<cudaStream_t>(stream));
    cudaStreamWaitEvent(p->capture, ready, 0);
    if (cudaMemcpyAsync(p->d_desc, descs, sizeof(cg_desc) * size_t(n), cudaMemcpyHostToDevice,
                        p->capture) != cudaSuccess)
      rc = CG_ECUDA;
    for (const Bin& b : p->bins)
      if (rc == CG_OK && !b.work.empty() &&
          cudaMemcpyAsync(p->d_work + b.work_off, b.work.data(), sizeof(int2) * b.work.size(),
                          cudaMemcpyHostToDevice, p->capture) != cudaSuccess)
        rc = CG_ECUDA;
    if (cudaStreamSynchronize(p->capture) != cudaSuccess && rc == CG_OK) rc = CG_ECUDA;
    cudaEventDestroy(ready);
  }
  // launch shapes (grid per bin: resident CTAs, at most one per work unit)
  for (Bin& b : p->bins) {
    if (rc != CG_OK) break;
    BatchArgs a{};
    a.n_work = int64_t(b.work.size());
    a.PB = b.PB;
    a.PR = b.PR;
    a.PEX = b.PEX;
    const int32_t prec = precision == CG_PREC_AUTO ? CG_PREC_FP16X3 : precision;
    const cudaError_t err = launch_batch_tc(b.op, b.UT, precision_el(prec), precision_x3(prec),
                                            b.full, a, 0, nullptr, false, nullptr, &b.grid);
    if (err != cudaSuccess) rc = err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  if (rc == CG_OK && !p->bins.empty()) {
    if (precision != CG_PREC_AUTO) {
      rc = capture(p, precision);
    } else {
      const std::string key = shape_key(p->bins, p->dev);
      int32_t chosen = -1;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) chosen = it->second.precision;
      }
      if (chosen < 0) {
        // time the accurate candidates on this batch (these runs write the outputs)
        float best = 1e30f;
        const int32_t cands[2] = {CG_PREC_FP16X3, CG_PREC_BF16X3};
        for (int32_t c : cands) {
          if (capture(p, c) != CG_OK) continue;
          const float ms = time_graph(p, 3);
          if (ms < best) {
            best = ms;
            chosen = c;
          }
        }
        if (chosen < 0) rc = CG_ECUDA;
        else {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tune[key] = Tuned{chosen};
        }
      }
      if (rc == CG_OK) rc = capture(p, chosen);
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
  if (precision) *precision = p->precision;
  if (n_bins) *n_bins = int32_t(p->bins.size());
  return CG_OK;
}

int cg_plan_destroy(cg_plan* p) {
  if (p == nullptr) return CG_EINVAL;
  destroy_plan(p);
  return CG_OK;
}

}  // extern "C"
