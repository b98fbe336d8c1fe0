// Host side of the serving loop behind cg_serve_*: ring slots, admission by
// HBM budget, stream-ordered publication into device memory (no host wait),
// on-demand launch of the persistent class kernels (liveness read from
// mapped memory, no CUDA call), completion polling and bounded shutdown.
#include <atomic>
#include <chrono>
#include <cstring>
#include <ctime>
#include <mutex>
#include <thread>
#include <vector>

#include "cgmimo.h"
#include "host_checks.h"
#include "launch.cuh"

using namespace cgm;

namespace {

constexpr int kClasses = 6;  // (detect, precode) x (UT 8, 16, 32)

int64_t mono_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return int64_t(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

// Class of a request: (operation, padded users 8 / 16 / 32). Detection with
// the exact tracker runs in the (detect, 32) class, whose CTA kernel has the
// shared memory for it; the 8- and 16-user classes run one warp per instance.
int class_of(const cg_desc& d, int* UT) {
  const int pu = padded_users(d.U);
  *UT = pu < 8 ? 8 : pu;
  if (d.op == CG_OP_DETECT && d.sinr_mode == CG_SINR_EXACT) *UT = 32;
  return d.op * 3 + (*UT == 8 ? 0 : *UT == 16 ? 1 : 2);
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
  bool released = true;  // its bytes no longer count against the budget
  bool reaped = true;    // a poll has reported it done: the slot may be reused
};

}  // namespace

struct cg_server {
  int dev = 0;
  cg_serve_cfg cfg{};
  int el = 1;
  bool x3 = true;
  // device memory: slot records, class heads, class tails, class rings
  void* dmem = nullptr;
  ServeSlot* d_slots = nullptr;
  unsigned long long* d_head = nullptr;
  unsigned long long* d_tail = nullptr;
  unsigned long long* d_ring = nullptr;
  // pinned staging of the asynchronous copies that publish a request
  void* smem_host = nullptr;
  ServeSlot* st_slot = nullptr;          // [cap] slot records
  unsigned long long* st_ring = nullptr;  // [classes][cap] ring entries
  unsigned long long* st_tail = nullptr;  // [cap] class tail published with each ticket
  // mapped host memory: control block and completion records
  void* hmem = nullptr;
  ServeCtrl* h_ctrl = nullptr;
  ServeCompletion* h_comp = nullptr;
  ServeCtrl* d_ctrl = nullptr;
  ServeCompletion* d_comp = nullptr;
  cudaStream_t ks[kClasses] = {};
  cudaStream_t cs = nullptr;
  unsigned long long launched_gen[kClasses] = {};
  int grid[kClasses] = {};
  std::mutex mu;
  uint64_t next = 0, head = 0;
  uint64_t published[kClasses] = {};
  std::vector<SlotInfo> info;
  int64_t inflight = 0;
};

namespace {

ServeArgs args_for(const cg_server* s, int cls) {
  ServeArgs a{};
  a.slots = s->d_slots;
  a.class_ring = s->d_ring;
  a.class_tail = s->d_tail;
  a.ctrl = s->d_ctrl;
  a.comp = s->d_comp;
  a.class_head = s->d_head;
  a.cls = cls;
  a.cap = s->cfg.capacity;
  a.PB = s->cfg.max_B;
  a.PR = s->cfg.max_R;
  a.PEX = cls == 2 ? 1 : 0;
  a.idle_ns = (unsigned long long)s->cfg.idle_timeout_ms * 1000000ull;
  a.gen = s->launched_gen[cls];
  return a;
}

int class_ut(int cls) { return cls % 3 == 0 ? 8 : cls % 3 == 1 ? 16 : 32; }

// Launches the class kernel unless a launch of it is still alive: the last
// work unit of launch generation g to exit writes g into the mapped control
// block, so the check is a memory read. A relaunch queues on the class
// stream behind a launch that is just finishing.
int ensure_running(cg_server* s, int cls) {
  const auto* ex = reinterpret_cast<const std::atomic<unsigned long long>*>(
      &s->h_ctrl->exited_gen[cls]);
  if (s->launched_gen[cls] > ex->load(std::memory_order_acquire)) return CG_OK;
  ++s->launched_gen[cls];
  const cudaError_t err = launch_serve_tc(cls / 3, class_ut(cls), s->el, s->x3, args_for(s, cls),
                                          s->grid[cls], s->ks[cls], true, nullptr, nullptr);
  if (err != cudaSuccess) {
    --s->launched_gen[cls];
    return CG_ECUDA;
  }
  return CG_OK;
}

bool complete(const cg_server* s, uint64_t ticket) {
  const ServeCompletion* c = s->h_comp + ticket % uint64_t(s->cfg.capacity);
  const auto* seq = reinterpret_cast<const std::atomic<unsigned long long>*>(&c->seq);
  return seq->load(std::memory_order_acquire) == ticket + 1;
}

// Releases the budget bytes of every completed request, then frees the
// ring slots at the head whose requests a poll has reported done.
void retire(cg_server* s) {
  const uint64_t cap = uint64_t(s->cfg.capacity);
  for (uint64_t t = s->head; t < s->next; ++t) {
    SlotInfo& in = s->info[t % cap];
    if (!in.released && complete(s, t)) {
      s->inflight -= in.bytes;
      in.released = true;
    }
  }
  while (s->head < s->next && s->info[s->head % cap].reaped) ++s->head;
}

void destroy_server(cg_server* s) {
  for (int c = 0; c < kClasses; ++c)
    if (s->ks[c]) cudaStreamDestroy(s->ks[c]);
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->dmem) cudaFree(s->dmem);
  if (s->hmem) cudaFreeHost(s->hmem);
  if (s->smem_host) cudaFreeHost(s->smem_host);
  delete s;
}

}  // namespace

extern "C" {

int cg_serve_create(const cg_serve_cfg* cfg, cg_server** out) {
  if (cfg == nullptr || out == nullptr) return CG_EINVAL;
  *out = nullptr;
  const cg_serve_cfg c = *cfg;
  if (c.capacity < 1 || c.capacity > (1 << 20)) return CG_EINVAL;
  if (c.precision < CG_PREC_BF16 || c.precision > CG_PREC_FP16X3) return CG_EINVAL;
  if (c.hbm_budget_bytes <= 0) return CG_EINVAL;
  if (c.max_B < 1 || c.max_B > CG_B_MAX || c.max_R < 1 || c.max_R > CG_R_MAX) return CG_EINVAL;
  if (c.ctas_per_class < 0 || c.idle_timeout_ms < 1 || c.idle_timeout_ms > 60000)
    return CG_EINVAL;
  cg_server* s = new cg_server();
  s->cfg = c;
  s->el = (c.precision == CG_PREC_BF16 || c.precision == CG_PREC_BF16X3) ? 0 : 1;
  s->x3 = c.precision == CG_PREC_BF16X3 || c.precision == CG_PREC_FP16X3;
  s->info.resize(size_t(c.capacity));
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return CG_ECUDA;
  }
  const size_t cap = size_t(c.capacity);
  const size_t u64 = sizeof(unsigned long long);
  const size_t head_off = sizeof(ServeSlot) * cap;
  const size_t tail_off = head_off + u64 * 8;
  const size_t ring_off = tail_off + u64 * 8;
  const size_t dbytes = ring_off + u64 * kClasses * cap;
  const size_t comp_off = (sizeof(ServeCtrl) + 255) & ~size_t(255);
  const size_t hbytes = comp_off + sizeof(ServeCompletion) * cap;
  const size_t st_ring_off = sizeof(ServeSlot) * cap;
  const size_t st_tail_off = st_ring_off + u64 * kClasses * cap;
  const size_t sbytes = st_tail_off + u64 * cap;
  int rc = CG_OK;
  if (cudaMalloc(&s->dmem, dbytes) != cudaSuccess) {
    s->dmem = nullptr;
    rc = CG_ENOMEM;
  }
  if (rc == CG_OK && cudaHostAlloc(&s->hmem, hbytes, cudaHostAllocMapped) != cudaSuccess) {
    s->hmem = nullptr;
    rc = CG_ENOMEM;
  }
  if (rc == CG_OK && cudaHostAlloc(&s->smem_host, sbytes, cudaHostAllocDefault) != cudaSuccess) {
    s->smem_host = nullptr;
    rc = CG_ENOMEM;
  }
  if (rc == CG_OK) {
    std::memset(s->hmem, 0, hbytes);
    std::memset(s->smem_host, 0, sbytes);
    char* dm = static_cast<char*>(s->dmem);
    s->d_slots = reinterpret_cast<ServeSlot*>(dm);
    s->d_head = reinterpret_cast<unsigned long long*>(dm + head_off);
    s->d_tail = reinterpret_cast<unsigned long long*>(dm + tail_off);
    s->d_ring = reinterpret_cast<unsigned long long*>(dm + ring_off);
    char* st = static_cast<char*>(s->smem_host);
    s->st_slot = reinterpret_cast<ServeSlot*>(st);
    s->st_ring = reinterpret_cast<unsigned long long*>(st + st_ring_off);
    s->st_tail = reinterpret_cast<unsigned long long*>(st + st_tail_off);
    char* h = static_cast<char*>(s->hmem);
    s->h_ctrl = reinterpret_cast<ServeCtrl*>(h);
    s->h_comp = reinterpret_cast<ServeCompletion*>(h + comp_off);
    void* dv = nullptr;
    if (cudaHostGetDevicePointer(&dv, s->hmem, 0) != cudaSuccess) rc = CG_ECUDA;
    char* d = static_cast<char*>(dv);
    s->d_ctrl = reinterpret_cast<ServeCtrl*>(d);
    s->d_comp = reinterpret_cast<ServeCompletion*>(d + comp_off);
  }
  if (rc == CG_OK && cudaMemset(s->dmem, 0, dbytes) != cudaSuccess) rc = CG_ECUDA;
  for (int k = 0; k < kClasses && rc == CG_OK; ++k)
    if (cudaStreamCreateWithFlags(&s->ks[k], cudaStreamNonBlocking) != cudaSuccess) rc = CG_ECUDA;
  if (rc == CG_OK && cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess)
    rc = CG_ECUDA;
  // launch shapes: each class gets a share of the SMs in proportion to the
  // cost of one of its instances (weights 1, 2, 8 for 8, 16, 32 padded
  // users), as many work units as are resident on that share
  DeviceInfo di;
  if (rc == CG_OK && device_info(&di) != 0) rc = CG_ECUDA;
  const double weight[3] = {1.0, 2.0, 8.0};
  const double wsum = 2.0 * (weight[0] + weight[1] + weight[2]);
  for (int k = 0; k < kClasses && rc == CG_OK; ++k) {
    uint32_t smem = 0;
    int resident = 0;
    const cudaError_t err = launch_serve_tc(k / 3, class_ut(k), s->el, s->x3, args_for(s, k), 0,
                                            nullptr, false, &smem, &resident);
    if (err != cudaSuccess) {
      rc = err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
      break;
    }
    const int share = int(double(resident) * weight[k % 3] / wsum + 0.5);
    s->grid[k] = c.ctas_per_class > 0 ? c.ctas_per_class : (share > 0 ? share : 1);
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
  if (uint64_t(d.n_inst) > SERVE_NINST_MASK) return CG_ETOOBIG;
  std::lock_guard<std::mutex> lk(s->mu);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->dev) return CG_EINVAL;
  retire(s);
  const uint64_t cap = uint64_t(s->cfg.capacity);
  if (s->next - s->head >= cap) return CG_EAGAIN;
  if (s->inflight + bytes > s->cfg.hbm_budget_bytes) return CG_EAGAIN;
  int UT;
  const int cls = class_of(d, &UT);
  const uint64_t t = s->next;
  const uint64_t slot = t % cap;
  if (t >> (64 - SERVE_NINST_BITS)) return CG_ETOOBIG;  // ticket space exhausted
  // publication: the slot record, the class ring entry and the new class
  // tail are copied in that order on one stream, so the device sees the
  // tail only after the record and the entry have landed. Each copy reads
  // its own pinned staging word (records and tails per slot, entries per
  // ring position), which stays unchanged until the copy has run.
  ServeSlot& rec = s->st_slot[slot];
  rec = ServeSlot{};
  rec.d = d;
  rec.ticket = t;
  rec.claim = (t & 0xffffffffull) << 32;
  std::memset(&s->h_comp[slot], 0, sizeof(ServeCompletion));
  const size_t pos = size_t(cls) * cap + size_t(s->published[cls] % cap);
  s->st_ring[pos] = (t << SERVE_NINST_BITS) | uint64_t(d.n_inst);
  s->st_tail[slot] = s->published[cls] + 1;
  if (cudaMemcpyAsync(s->d_slots + slot, &rec, sizeof(rec), cudaMemcpyHostToDevice, s->cs) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->d_ring + pos, &s->st_ring[pos], sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, s->cs) != cudaSuccess ||
      cudaMemcpyAsync(s->d_tail + cls, &s->st_tail[slot], sizeof(unsigned long long),
                      cudaMemcpyHostToDevice, s->cs) != cudaSuccess)
    return CG_ECUDA;
  ++s->published[cls];
  SlotInfo& in = s->info[slot];
  in.ticket = t;
  in.cls = cls;
  in.bytes = bytes;
  in.submit_ns = mono_ns();
  in.complete_ns = 0;
  in.released = false;
  in.reaped = false;
  s->inflight += bytes;
  s->next = t + 1;
  *ticket = t;
  return ensure_running(s, cls);
}

int cg_serve_poll(cg_server* s, uint64_t ticket, int32_t* done, cg_req_stats* stats) {
  if (s == nullptr || done == nullptr) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const uint64_t cap = uint64_t(s->cfg.capacity);
  SlotInfo& in = s->info[ticket % cap];
  if (ticket >= s->next || in.ticket != ticket) return CG_EINVAL;
  *done = complete(s, ticket) ? 1 : 0;
  if (*done) {
    if (in.complete_ns == 0) in.complete_ns = mono_ns();
    in.reaped = true;
    if (stats) {
      const ServeCompletion* c = s->h_comp + ticket % cap;
      stats->status = c->status;
      stats->pad = 0;
      stats->submit_ns = in.submit_ns;
      stats->complete_ns = in.complete_ns;
      stats->device_first_ns = int64_t(c->t_first_ns);
      stats->device_done_ns = int64_t(c->t_done_ns);
    }
    retire(s);
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
  for (int k = 0; k < kClasses; ++k) {
    while (s->launched_gen[k] > 0) {
      const cudaError_t q = cudaStreamQuery(s->ks[k]);
      if (q != cudaErrorNotReady) break;
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10)) return CG_ETIMEDOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  if (cudaStreamSynchronize(s->cs) != cudaSuccess) return CG_ECUDA;
  destroy_server(s);
  return CG_OK;
}

}  // extern "C"
