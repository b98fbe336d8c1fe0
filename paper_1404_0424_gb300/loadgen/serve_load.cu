// Load generator for the serving API: Poisson arrivals of uneven detection
// and precoding requests, submitted through the public C ABI either to a
// cg_server ("served") or as one cg_detect / cg_precode launch per request
// on one stream ("plain"). Latency is measured from each request's
// scheduled arrival to the host seeing it complete. Prints one JSON line.
//
// Request mix (seeded): operation 50/50, B in {64, 128, 256}, U in
// {8, 16, 32}, 16/64/256-QAM, subcarriers uniform 12..1200, symbols uniform
// 1..14, SNR uniform 5..25 dB, K = min(U/4, 8). Inputs are views at random
// offsets into a device pool of synthetic complex values; outputs go to a
// ring of per-request regions.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "cgmimo.h"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Synthetic pool values: a counter-based hash mapped to [-1, 1).
__global__ void fill_pool(float* p, size_t n, uint32_t seed) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    uint32_t x = uint32_t(i) * 2654435761u ^ seed ^ uint32_t(i >> 32) * 40503u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    p[i] = float(x) * (2.0f / 4294967296.0f) - 1.0f;
  }
}

struct Req {
  cg_desc d;
  int64_t arrival_ns;  // scheduled, relative to the start
  int64_t solves;
};

double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t k = std::min(v.size() - 1, size_t(p * (v.size() - 1) + 0.5));
  return v[k];
}

}  // namespace

int main(int argc, char** argv) {
  double rate = 20000.0, seconds = 2.0, pool_gb = 2.0;
  int capacity = 64, precision = CG_PREC_FP16X3, seed = 1;
  double budget_gb = 40.0;
  std::string mode = "served";
  for (int i = 1; i + 1 < argc; i += 2) {
    const std::string k = argv[i];
    const char* v = argv[i + 1];
    if (k == "--rate") rate = atof(v);
    else if (k == "--seconds") seconds = atof(v);
    else if (k == "--pool-gb") pool_gb = atof(v);
    else if (k == "--capacity") capacity = atoi(v);
    else if (k == "--precision") precision = atoi(v);
    else if (k == "--seed") seed = atoi(v);
    else if (k == "--budget-gb") budget_gb = atof(v);
    else if (k == "--mode") mode = v;
  }
  const bool served = mode == "served";

  // ---- request schedule
  std::mt19937_64 rng{static_cast<uint64_t>(seed)};
  std::exponential_distribution<double> gap(rate);
  std::uniform_int_distribution<int> pick3(0, 2), nsc(12, 1200), rsym(1, 14), op2(0, 1);
  std::uniform_real_distribution<double> snr(5.0, 25.0);
  const int Bs[3] = {64, 128, 256}, Us[3] = {8, 16, 32}, Qs[3] = {4, 6, 8};
  std::vector<Req> reqs;
  double t = 0.0;
  while (t < seconds) {
    t += gap(rng);
    Req r{};
    r.d.op = op2(rng);
    r.d.B = Bs[pick3(rng)];
    r.d.U = Us[pick3(rng)];
    r.d.qam_bits = Qs[pick3(rng)];
    r.d.n_inst = nsc(rng);
    r.d.R = rsym(rng);
    r.d.K = std::max(1, std::min(r.d.U / 4, 8));
    r.d.Es = 1.0f;
    r.d.N0 = float(r.d.U / std::pow(10.0, snr(rng) / 10.0));
    r.d.sinr_mode = 0;
    r.arrival_ns = int64_t(t * 1e9);
    r.solves = r.d.n_inst * r.d.R;
    reqs.push_back(r);
  }

  // ---- device pool (inputs) and output ring
  const size_t pool_floats = size_t(pool_gb * (1 << 30)) / sizeof(float) & ~size_t(3);
  float* pool = nullptr;
  // largest output region in bytes: q of a 1200 x 14 x 256 precode request plus
  // its norms and status words (detection outputs are smaller)
  const size_t max_out = size_t(1200) * 14 * 256 * 8 + size_t(1200) * 14 * 4 + 1200 * 4 + 1024;
  char* outs = nullptr;
  if (cudaMalloc(&pool, pool_floats * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&outs, max_out * size_t(capacity)) != cudaSuccess) {
    printf("{\"error\": \"allocation failed\"}\n");
    return 1;
  }
  fill_pool<<<1024, 256>>>(pool, pool_floats, uint32_t(seed) * 977u);
  cudaDeviceSynchronize();
  std::uniform_int_distribution<size_t> off(0, 1ull << 62);
  for (Req& r : reqs) {
    const size_t hn = size_t(r.d.n_inst) * r.d.B * r.d.U * 2;
    const size_t in_n = size_t(r.d.n_inst) * r.d.R * (r.d.op == 0 ? r.d.B : r.d.U) * 2;
    r.d.H = pool + (off(rng) % (pool_floats - hn)) / 4 * 4;
    r.d.in = pool + (off(rng) % (pool_floats - in_n)) / 4 * 4;
  }

  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cg_server* srv = nullptr;
  if (served) {
    cg_serve_cfg cfg{};
    cfg.capacity = capacity;
    cfg.precision = precision;
    cfg.hbm_budget_bytes = int64_t(budget_gb * (1ll << 30));
    cfg.max_B = 256;
    cfg.max_R = 14;
    cfg.ctas_per_class = 0;
    cfg.idle_timeout_ms = 2000;
    const int rc = cg_serve_create(&cfg, &srv);
    if (rc != CG_OK) {
      printf("{\"error\": \"cg_serve_create: %s\"}\n", cg_strerror(rc));
      return 1;
    }
  }
  std::vector<cudaEvent_t> evs(static_cast<size_t>(capacity));
  for (auto& e : evs) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);

  struct Flight {
    size_t req;
    uint64_t ticket;
    int region;
  };
  std::vector<Flight> flight;
  std::vector<int> free_regions;
  for (int k = capacity - 1; k >= 0; --k) free_regions.push_back(k);
  std::vector<double> lat_ms, svc_ms;  // latency from arrival; device service time (served)
  int64_t loops = 0, submit_ns = 0, poll_ns = 0;
  std::vector<double> cls_lat[6];  // (operation, padded users 8 / 16 / 32)
  auto cls_of = [](const cg_desc& d) {
    return d.op * 3 + (d.U <= 8 ? 0 : d.U <= 16 ? 1 : 2);
  };
  int64_t solves_done = 0, eagain = 0;
  size_t next = 0, max_inflight = 0;
  const int64_t t0 = now_ns();
  const int64_t deadline = t0 + int64_t((seconds + 20.0) * 1e9);
  int64_t last_done = t0;

  auto set_outputs = [&](cg_desc& d, int region) {
    char* base = outs + size_t(region) * max_out;
    const size_t ru = size_t(d.n_inst) * d.R * d.U;
    if (d.op == 0) {
      d.out = base;
      d.mu = reinterpret_cast<float*>(base + ru * 8);
      d.rho = reinterpret_cast<float*>(base + ru * 12);
      d.aux = reinterpret_cast<float*>(base + ru * 16);
      d.status = reinterpret_cast<int32_t*>(base + ru * (16 + 4 * d.qam_bits));
    } else {
      const size_t rb = size_t(d.n_inst) * d.R * d.B;
      d.out = base;
      d.mu = d.rho = nullptr;
      d.aux = reinterpret_cast<float*>(base + rb * 8);
      d.status = reinterpret_cast<int32_t*>(base + rb * 8 + size_t(d.n_inst) * d.R * 4 + 16);
    }
  };

  while ((next < reqs.size() || !flight.empty()) && now_ns() < deadline) {
    const int64_t now = now_ns() - t0;
    ++loops;
    const int64_t ts0 = now_ns();
    // submit every request that is due, while a region is free
    while (next < reqs.size() && reqs[next].arrival_ns <= now && !free_regions.empty()) {
      Req& r = reqs[next];
      const int region = free_regions.back();
      set_outputs(r.d, region);
      uint64_t ticket = 0;
      int rc;
      if (served) {
        rc = cg_serve_submit(srv, &r.d, &ticket);
        if (rc == CG_EAGAIN) {
          ++eagain;
          break;
        }
      } else {
        cg_params p{};
        p.B = r.d.B;
        p.U = r.d.U;
        p.qam_bits = r.d.qam_bits;
        p.K = r.d.K;
        p.R = r.d.R;
        p.N0 = r.d.N0;
        p.Es = r.d.Es;
        p.precision = CG_PREC_FP32;
        rc = r.d.op == 0 ? cg_detect(&p, r.d.n_inst, r.d.H, r.d.in, r.d.out, r.d.mu, r.d.rho,
                                     r.d.aux, r.d.status, st)
                         : cg_precode(&p, r.d.n_inst, r.d.H, r.d.in, r.d.out, r.d.aux, 0,
                                      r.d.status, st);
        if (rc == CG_OK) rc = cudaEventRecord(evs[size_t(region)], st) == cudaSuccess ? CG_OK : CG_ECUDA;
      }
      if (rc != CG_OK) {
        printf("{\"error\": \"submit: %s\", \"op\": %d, \"B\": %d, \"U\": %d, \"R\": %d, "
               "\"K\": %d, \"n\": %lld}\n",
               cg_strerror(rc), r.d.op, r.d.B, r.d.U, r.d.R, r.d.K, (long long)r.d.n_inst);
        return 1;
      }
      free_regions.pop_back();
      flight.push_back(Flight{next, ticket, region});
      max_inflight = std::max(max_inflight, flight.size());
      ++next;
    }
    const int64_t ts1 = now_ns();
    submit_ns += ts1 - ts0;
    // completions
    for (size_t k = 0; k < flight.size();) {
      const Flight f = flight[k];
      bool done = false;
      if (served) {
        int32_t dn = 0;
        cg_req_stats s{};
        if (cg_serve_poll(srv, f.ticket, &dn, &s) != CG_OK) {
          printf("{\"error\": \"poll failed\"}\n");
          return 1;
        }
        done = dn != 0;
        if (done) svc_ms.push_back(double(s.device_done_ns - s.device_first_ns) * 1e-6);
      } else {
        done = cudaEventQuery(evs[size_t(f.region)]) == cudaSuccess;
      }
      if (done) {
        const int64_t tdone = now_ns();
        lat_ms.push_back(double(tdone - t0 - reqs[f.req].arrival_ns) * 1e-6);
        cls_lat[cls_of(reqs[f.req].d)].push_back(lat_ms.back());
        solves_done += reqs[f.req].solves;
        last_done = tdone;
        free_regions.push_back(f.region);
        flight[k] = flight.back();
        flight.pop_back();
      } else {
        ++k;
      }
    }
    poll_ns += now_ns() - ts1;
    // both modes poll without sleeping: a sleep of a few microseconds lasts
    // the kernel's timer slack (tens of microseconds) and would delay the
    // moment a completion is seen
  }
  const double elapsed = double(last_done - t0) * 1e-9;
  if (srv) cg_serve_destroy(srv);
  cudaStreamSynchronize(st);
  double mean = 0;
  for (double v : lat_ms) mean += v;
  mean = lat_ms.empty() ? 0 : mean / lat_ms.size();
  std::string per_class = "{";
  const char* names[6] = {"detect8", "detect16", "detect32", "precode8", "precode16", "precode32"};
  for (int c = 0; c < 6; ++c) {
    char buf[160];
    snprintf(buf, sizeof(buf), "%s\"%s\": [%zu, %.4f, %.4f]", c ? ", " : "", names[c],
             cls_lat[c].size(), pct(cls_lat[c], 0.5), pct(cls_lat[c], 0.99));
    per_class += buf;
  }
  per_class += "}";
  printf("{\"mode\": \"%s\", \"requests\": %zu, \"completed\": %zu, \"offered_rps\": %.1f, "
         "\"achieved_rps\": %.1f, \"solves_per_s\": %.1f, \"lat_p50_ms\": %.4f, "
         "\"lat_p99_ms\": %.4f, \"lat_mean_ms\": %.4f, \"max_inflight\": %zu, \"eagain\": %lld, "
         "\"precision\": %d, \"per_class_count_p50_p99_ms\": %s, "
         "\"device_service_p50_p99_ms\": [%.4f, %.4f], \"host_loops\": %lld, "
         "\"host_submit_s\": %.3f, \"host_poll_s\": %.3f}\n",
         mode.c_str(), reqs.size(), lat_ms.size(), reqs.size() / seconds,
         lat_ms.size() / std::max(elapsed, 1e-9), solves_done / std::max(elapsed, 1e-9),
         pct(lat_ms, 0.5), pct(lat_ms, 0.99), mean, max_inflight, (long long)eagain,
         served ? precision : 0, per_class.c_str(), pct(svc_ms, 0.5), pct(svc_ms, 0.99),
         (long long)loops, submit_ns * 1e-9, poll_ns * 1e-9);
  return lat_ms.size() == reqs.size() ? 0 : 2;
}
