// Host side of the serving loop behind cg_serve_*: slots from a free list,
// admission by HBM budget, publication through mapped host memory with no
// CUDA call (a submit is a few stores and a release fence), on-demand launch
// of the persistent serving kernel (liveness read from mapped memory),
// completion polling and bounded shutdown.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <ctime>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "cgmimo.h"
#include "host_checks.h"
#include "cg_serve.cuh"
#include "launch.cuh"

using namespace cgm;

namespace {

// (detect, precode) x (UT 8, 16, 32) and exact-tracker detection with 8, 16
// or 32 padded users, all on the warp-per-instance serving kernel
constexpr int kClasses = kWarpClasses;
static_assert(kClasses <= kServeMaxClasses, "class count of the control block");
constexpr int kRingPerSlot = 4;   // class ring positions per slot (ring = 4 x capacity)
// One serving kernel; its liveness counters in the control block are those
// of its ServeArgs::cls.
constexpr int kKernels = 1;
int kernel_of(int) { return 0; }
int live_index(int) { return 0; }

int64_t mono_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return int64_t(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

// Class of a request: (operation, padded users 8 / 16 / 32), one warp per
// instance; detection with the exact tracker (Eq. 10) has classes 6, 7, 8
// for 8, 16, 32 padded users (the kernels of single calls and plans).
int class_of(const cg_desc& d, int* UT) {
  const int pu = padded_users(d.U);
  *UT = pu < 8 ? 8 : pu;
  const int uti = *UT == 8 ? 0 : *UT == 16 ? 1 : 2;
  if (d.op == CG_OP_DETECT && d.sinr_mode == CG_SINR_EXACT) return 6 + uti;
  return d.op * 3 + uti;
}


int64_t footprint(const cg_desc& d) {
  const int64_t n = d.n_inst, B = d.B, U = d.U, R = d.R, q = d.qam_bits;
  if (d.op == CG_OP_DETECT) return n * ((B * U + R * B) * 8 + R * U * (16 + 4 * q) + 4);
  return n * ((B * U + R * U) * 8 + R * B * 8 + R * 4 + 4);
}

struct SlotInfo {
  uint64_t ticket = ~0ull;
  int cls = 0;
  int64_t bytes = 0;
  int64_t submit_ns = 0;
  int64_t complete_ns = 0;
  bool in_use = false;   // holds a request that a poll has not yet reported done
  bool released = true;  // its bytes no longer count against the budget
};

}  // namespace

struct cg_server {
  int dev = 0;
  cg_serve_cfg cfg{};
  int el = 1;
  bool x3 = true;
  int cap = 0, ring = 0;
  // device memory: per-slot progress counters, class heads
  void* dmem = nullptr;
  ServeCount* d_counts = nullptr;
  ServeMirror* d_mirror = nullptr;
  unsigned long long* d_head = nullptr;
  // mapped host memory: control block, completions, descriptors, class rings
  void* hmem = nullptr;
  ServeCtrl* h_ctrl = nullptr;
  ServeCompletion* h_comp = nullptr;
  ServeDesc* h_desc = nullptr;
  ServeEntry* h_ring = nullptr;
  ServeCtrl* d_ctrl = nullptr;
  ServeCompletion* d_comp = nullptr;
  ServeDesc* d_desc = nullptr;
  ServeEntry* d_ring = nullptr;
  cudaStream_t ks[kKernels] = {};
  unsigned long long launched_gen[kKernels] = {};
  int grid[kKernels] = {};
  std::mutex mu;
  uint64_t next = 0;                                 // next ticket
  uint64_t published[kClasses] = {};
  uint64_t published_total = 0;
  std::deque<std::pair<uint64_t, int>> queued[kClasses];  // (ticket, slot) not yet seen complete
  std::vector<int> free_slots;
  std::vector<SlotInfo> info;                        // per slot
  std::unordered_map<uint64_t, int> ticket_slot;     // slot of each ticket that holds one
  int64_t inflight = 0;                              // budget bytes of unfinished requests
};

namespace {

ServeArgs args_for(const cg_server* s, int k) {
  ServeArgs a{};
  a.counts = s->d_counts;
  a.mirror = s->d_mirror;
  a.descs = s->d_desc;
  a.class_ring = s->d_ring;
  a.ctrl = s->d_ctrl;
  a.comp = s->d_comp;
  a.class_head = s->d_head;
  a.cls = live_index(k);
  a.cap = s->ring;
  a.PB = s->cfg.max_B;
  a.PR = s->cfg.max_R;
  a.PEX = 0;
  a.poll_host = 1;
  a.idle_ns = (unsigned long long)s->cfg.idle_timeout_ms * 1000000ull;
  a.gen = s->launched_gen[k];
  return a;
}

// Launches serving kernel k (or, with launch = false, reports its resident CTAs).
cudaError_t launch_kernel(const cg_server* s, int k, bool launch, int* resident) {
  const ServeArgs a = args_for(s, k);
  return launch_serve_warp(s->el, s->x3, a, s->grid[k], s->ks[k], launch, resident);
}

// Launches the serving kernel of a class unless a launch of it is still
// alive: the last work unit of launch generation g to exit writes g into the
// mapped control block, so the check is a memory read. A relaunch queues on
// the kernel's stream behind a launch that is just finishing.
int ensure_running(cg_server* s, int cls) {
  const int k = kernel_of(cls);
  const auto* ex = reinterpret_cast<const std::atomic<unsigned long long>*>(
      &s->h_ctrl->exited_gen[live_index(k)]);
  if (s->launched_gen[k] > ex->load(std::memory_order_acquire)) return CG_OK;
  ++s->launched_gen[k];
  if (launch_kernel(s, k, true, nullptr) != cudaSuccess) {
    --s->launched_gen[k];
    return CG_ECUDA;
  }
  return CG_OK;
}

bool complete(const cg_server* s, uint64_t ticket, int slot) {
  const auto* seq =
      reinterpret_cast<const std::atomic<unsigned long long>*>(&s->h_comp[slot].seq);
  return seq->load(std::memory_order_acquire) == ticket + 1;
}

// Releases the budget bytes of completed requests and drops completed
// requests from the front of the class queues (a class ring position is
// reused only after its request is complete, hence fully handed out).
void retire(cg_server* s) {
  for (int sl = 0; sl < s->cap; ++sl) {
    SlotInfo& in = s->info[sl];
    if (in.in_use && !in.released && complete(s, in.ticket, sl)) {
      s->inflight -= in.bytes;
      in.released = true;
    }
  }
  for (int c = 0; c < kClasses; ++c) {
    auto& q = s->queued[c];
    while (!q.empty()) {
      const uint64_t t = q.front().first;
      const int sl = q.front().second;
      if (s->info[sl].ticket == t && !complete(s, t, sl)) break;
      q.pop_front();
    }
  }
}

void destroy_server(cg_server* s) {
  for (int k = 0; k < kKernels; ++k)
    if (s->ks[k]) cudaStreamDestroy(s->ks[k]);
  if (s->dmem) cudaFree(s->dmem);
  if (s->hmem) cudaFreeHost(s->hmem);
  delete s;
}

}  // namespace

extern "C" {

int cg_serve_create(const cg_serve_cfg* cfg, cg_server** out) {
  if (cfg == nullptr || out == nullptr) return CG_EINVAL;
  *out = nullptr;
  const cg_serve_cfg c = *cfg;
  if (c.capacity < 1 || c.capacity > (1 << 14)) return CG_EINVAL;
  if (c.precision < CG_PREC_BF16 || c.precision > CG_PREC_FP16X3) return CG_EINVAL;
  if (c.hbm_budget_bytes <= 0) return CG_EINVAL;
  if (c.max_B < 1 || c.max_B > CG_B_MAX || c.max_R < 1 || c.max_R > CG_R_MAX) return CG_EINVAL;
  if (c.ctas_per_class < 0 || c.idle_timeout_ms < 1 || c.idle_timeout_ms > 60000)
    return CG_EINVAL;
  cg_server* s = new cg_server();
  s->cfg = c;
  s->el = (c.precision == CG_PREC_BF16 || c.precision == CG_PREC_BF16X3) ? 0 : 1;
  s->x3 = c.precision == CG_PREC_BF16X3 || c.precision == CG_PREC_FP16X3;
  s->cap = c.capacity;
  s->ring = kRingPerSlot * c.capacity;
  s->info.resize(size_t(s->cap));
  s->ticket_slot.reserve(size_t(s->cap) * 2);
  for (int sl = s->cap - 1; sl >= 0; --sl) s->free_slots.push_back(sl);
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return CG_ECUDA;
  }
  const size_t cap = size_t(s->cap);
  const size_t positions = size_t(kClasses) * size_t(s->ring);
  const size_t mirror_off = (sizeof(ServeCount) * positions + 255) & ~size_t(255);
  const size_t head_off = mirror_off + sizeof(ServeMirror) * positions;
  const size_t dbytes = head_off + sizeof(unsigned long long) * kServeHeadWords;
  const size_t comp_off = (sizeof(ServeCtrl) + 255) & ~size_t(255);
  const size_t desc_off = comp_off + sizeof(ServeCompletion) * cap;
  const size_t ring_off = desc_off + sizeof(ServeDesc) * cap;
  const size_t hbytes = ring_off + sizeof(ServeEntry) * kClasses * size_t(s->ring);
  int rc = CG_OK;
  if (cudaMalloc(&s->dmem, dbytes) != cudaSuccess) {
    s->dmem = nullptr;
    rc = CG_ENOMEM;
  }
  if (rc == CG_OK && cudaHostAlloc(&s->hmem, hbytes, cudaHostAllocMapped) != cudaSuccess) {
    s->hmem = nullptr;
    rc = CG_ENOMEM;
  }
  if (rc == CG_OK) {
    std::memset(s->hmem, 0, hbytes);
    char* dm = static_cast<char*>(s->dmem);
    s->d_counts = reinterpret_cast<ServeCount*>(dm);
    s->d_mirror = reinterpret_cast<ServeMirror*>(dm + mirror_off);
    s->d_head = reinterpret_cast<unsigned long long*>(dm + head_off);
    char* h = static_cast<char*>(s->hmem);
    s->h_ctrl = reinterpret_cast<ServeCtrl*>(h);
    s->h_comp = reinterpret_cast<ServeCompletion*>(h + comp_off);
    s->h_desc = reinterpret_cast<ServeDesc*>(h + desc_off);
    s->h_ring = reinterpret_cast<ServeEntry*>(h + ring_off);
    void* dv = nullptr;
    if (cudaHostGetDevicePointer(&dv, s->hmem, 0) != cudaSuccess) rc = CG_ECUDA;
    char* d = static_cast<char*>(dv);
    s->d_ctrl = reinterpret_cast<ServeCtrl*>(d);
    s->d_comp = reinterpret_cast<ServeCompletion*>(d + comp_off);
    s->d_desc = reinterpret_cast<ServeDesc*>(d + desc_off);
    s->d_ring = reinterpret_cast<ServeEntry*>(d + ring_off);
  }
  if (rc == CG_OK && (cudaMemset(s->dmem, 0, dbytes) != cudaSuccess ||
                      cudaDeviceSynchronize() != cudaSuccess))
    rc = CG_ECUDA;
  for (int k = 0; k < kKernels && rc == CG_OK; ++k)
    if (cudaStreamCreateWithFlags(&s->ks[k], cudaStreamNonBlocking) != cudaSuccess) rc = CG_ECUDA;
  // launch shape: every serving CTA fills one SM (its shared memory is
  // padded past half an SM), one CTA on every SM
  DeviceInfo di;
  if (rc == CG_OK && device_info(&di) != 0) rc = CG_ECUDA;
  if (rc == CG_OK) {
    s->grid[0] = di.sm_count;
    if (c.ctas_per_class > 0) s->grid[0] = std::min(s->grid[0], c.ctas_per_class);
  }
  for (int k = 0; k < kKernels && rc == CG_OK; ++k) {
    int resident = 0;
    const cudaError_t err = launch_kernel(s, k, false, &resident);
    if (err != cudaSuccess)
      rc = err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
    else if (resident > di.sm_count)  // the padding did not make it one CTA per SM
      rc = CG_ECUDA;
  }
  if (rc != CG_OK) {
    destroy_server(s);
    return rc;
  }
  *out = s;
  return CG_OK;
}

int cg_serve_submit(cg_server* s, const cg_desc* req, uint64_t* ticket) {
  if (s == nullptr || req == nullptr || ticket == nullptr) return CG_EINVAL;
  const cg_desc d = *req;
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
  p.precision = s->cfg.precision;
  if (d.n_inst < 1 || d.B > s->cfg.max_B || d.R > s->cfg.max_R) return CG_EINVAL;
  int rc;
  if (d.op == CG_OP_DETECT)
    rc = check_detect(&p, d.n_inst, d.H, d.in, d.out, d.mu, d.rho, d.aux, d.status);
  else if (d.op == CG_OP_PRECODE)
    rc = check_precode(&p, d.n_inst, d.H, d.in, d.out, d.aux, d.status);
  else
    rc = CG_EINVAL;
  if (rc != CG_OK) return rc;
  const int64_t bytes = footprint(d);
  if (bytes > s->cfg.hbm_budget_bytes) return CG_ETOOBIG;
  if (d.n_inst >= (int64_t(1) << 24)) return CG_ETOOBIG;  // 24-bit instance counts
  std::lock_guard<std::mutex> lk(s->mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->dev) return CG_EINVAL;
  retire(s);
  int UT;
  const int cls = class_of(d, &UT);
  if (s->free_slots.empty()) return CG_EAGAIN;
  if (s->inflight + bytes > s->cfg.hbm_budget_bytes) return CG_EAGAIN;
  if (s->queued[cls].size() >= size_t(s->ring)) return CG_EAGAIN;
  const int slot = s->free_slots.back();
  s->free_slots.pop_back();
  if (s->info[slot].ticket != ~0ull) s->ticket_slot.erase(s->info[slot].ticket);
  const uint64_t t = s->next++;
  // publication: descriptor, completion record and ring entry first, then
  // (release) the class tail that makes them visible to the class kernel
  ServeDesc& ds = s->h_desc[slot];
  ds.d = d;
  ds.ticket = t;
  std::memset(&s->h_comp[slot], 0, sizeof(ServeCompletion));
  ServeEntry& e = s->h_ring[size_t(cls) * s->ring + size_t(s->published[cls] % s->ring)];
  e.slot_ninst = (uint64_t(slot) << 32) | uint64_t(d.n_inst);
  e.ticket = t;
  ++s->published[cls];
  ++s->published_total;
  std::atomic_thread_fence(std::memory_order_release);
  reinterpret_cast<std::atomic<unsigned long long>*>(&s->h_ctrl->class_tail[cls])
      ->store(s->published[cls], std::memory_order_release);
  reinterpret_cast<std::atomic<unsigned long long>*>(&s->h_ctrl->class_tail[kServeTotal])
      ->store(s->published_total, std::memory_order_release);
  SlotInfo& in = s->info[slot];
  in.ticket = t;
  in.cls = cls;
  in.bytes = bytes;
  in.submit_ns = mono_ns();
  in.complete_ns = 0;
  in.in_use = true;
  in.released = false;
  s->inflight += bytes;
  s->queued[cls].emplace_back(t, slot);
  s->ticket_slot[t] = slot;
  *ticket = t;
  return ensure_running(s, cls);
}

int cg_serve_poll(cg_server* s, uint64_t ticket, int32_t* done, cg_req_stats* stats) {
  if (s == nullptr || done == nullptr) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket >= s->next) return CG_EINVAL;
  const auto found = s->ticket_slot.find(ticket);
  if (found == s->ticket_slot.end()) return CG_EINVAL;  // its slot serves a later request now
  const int slot = found->second;
  SlotInfo& in = s->info[slot];
  *done = (!in.in_use || complete(s, ticket, slot)) ? 1 : 0;
  if (*done) {
    if (in.complete_ns == 0) in.complete_ns = mono_ns();
    if (stats) {
      const ServeCompletion* c = s->h_comp + slot;
      stats->status = c->status;
      stats->pad = 0;
      stats->submit_ns = in.submit_ns;
      stats->complete_ns = in.complete_ns;
      stats->device_first_ns = int64_t(c->t_first_ns);
      stats->device_done_ns = int64_t(c->t_done_ns);
    }
    if (in.in_use) {  // first report of done: the slot becomes free
      if (!in.released) {
        s->inflight -= in.bytes;
        in.released = true;
      }
      in.in_use = false;
      s->free_slots.push_back(slot);
    }
    return CG_OK;
  }
  // not done: make sure its class kernel is alive (it may have idled out just
  // before the request was published)
  return ensure_running(s, in.cls);
}

int cg_serve_destroy(cg_server* s) {
  if (s == nullptr) return CG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    reinterpret_cast<std::atomic<int>*>(&s->h_ctrl->stop)->store(1, std::memory_order_release);
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < kKernels; ++k) {
    while (s->launched_gen[k] > 0) {
      const cudaError_t q = cudaStreamQuery(s->ks[k]);
      if (q != cudaErrorNotReady) break;
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10)) return CG_ETIMEDOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  destroy_server(s);
  return CG_OK;
}

}  // extern "C"
