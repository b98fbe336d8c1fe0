// Serving: requests published by the host through mapped host memory and
// claimed instance by instance by persistent kernels (cg_serve_*).
//
// Work units take their instances through the same warp-per-instance bodies
// as the single calls and the batched plans, with ServeArgs as their work
// source.
#pragma once

#include "cg_warp.cuh"


namespace cgm {

// ---------------------------------------------------------------------------
// Serving: requests published by the host, claimed instance by instance
// ---------------------------------------------------------------------------

// Serving protocol. The host publishes a request without any CUDA call:
// it writes the request's descriptor into its slot and the class ring entry
// (slot, instance count, ticket) into mapped host memory, then, after a
// release fence, the new class tail. The first work unit to need the
// request reads the tail with an acquire load, then the entry and the
// descriptor, and copies both into device memory (ServeMirror); all other
// work on the request reads that copy, so the link to host memory carries
// a few words per request rather than per instance. A request's progress
// lives in device memory, in two words of its class-ring position tagged
// with the low 32 bits of its ticket: the first unit to see an older tag
// starts the count afresh (compare-and-swap), so the host never resets
// device memory; every later unit counts with a plain atomicAdd, so claims
// do not serialise behind a compare-and-swap loop when hundreds of warps
// take instances of one request. A ring position is given to a new request
// only after 4 x capacity later requests of its class have been published
// (and its own request has completed), so the tag a unit has just read is
// still the one its atomicAdd lands on. Tickets grow by one per request, so
// tags compare by the sign of their 32-bit difference.

// Descriptor of the request in a slot (mapped host memory, host-written).
struct ServeDesc {
  cg_desc d;
  unsigned long long ticket;
};

// Progress of the request at a class-ring position (device memory).
//   claim: tag << 32 | next instance to hand out
//   done:  tag << 32 | instances finished << 8 | OR of their status words
struct ServeCount {
  unsigned long long claim;
  unsigned long long done;
};

// A published request in a class ring (mapped host memory).
struct ServeEntry {
  unsigned long long slot_ninst;  // slot << 32 | instance count
  unsigned long long ticket;
};

// Completion record in mapped host memory, written by the device.
struct ServeCompletion {
  unsigned long long seq;  // ticket + 1 once the request is complete
  unsigned long long t_first_ns, t_done_ns;  // device global timer
  int status;
  int pad;
};

// class_tail index of the total over all classes (host-written); the same
// index of the device head array holds the device's copy of that total, and
// kServeStop a device copy of the stop flag.
constexpr int kServeMaxClasses = 14;  // classes 0..13 may be used
constexpr int kServeTotal = 15;
constexpr int kServeStop = 14;
constexpr int kServeHeadWords = 16;

// Control block in mapped host memory: the stop flag and the class tails
// (host-written), and per serving kernel the number of running work units
// (CTAs or warps) and the launch generation whose last unit has exited
// (device-written), which let the host see whether a kernel is alive
// without a CUDA call.

struct ServeCtrl {
  unsigned long long class_tail[16];  // requests published per class; [15]: all classes
  int stop;
  int pad;
  int live[16];
  unsigned long long exited_gen[16];
};

// Threads of a serving CTA of the warp-per-instance kernels (8 warps: one
// such CTA fills an SM's share of the serving grid).
constexpr int kServeThreads = 256;

// Device copy of a published request, one per class-ring position: its
// descriptor and ring entry, valid when seq is the class sequence number of
// the request plus one. The first unit that needs the request and finds the
// copy missing reads the mapped host memory once and writes it (several
// units may race to write the same values); every other claim, descriptor
// read and completion of the request then stays in device memory.
struct __align__(16) ServeMirror {
  cg_desc d;
  unsigned long long slot_ninst;
  unsigned long long ticket;
  unsigned long long seq;
  unsigned long long pad;
};

struct ServeArgs {
  ServeCount* counts;           // device, one per class-ring position
  ServeMirror* mirror;          // device, one per class-ring position
  const ServeDesc* descs;       // mapped host, one per slot
  const ServeEntry* class_ring; // mapped host: [class][cap] published entries
  ServeCtrl* ctrl;              // mapped host
  ServeCompletion* comp;        // mapped host, one per slot
  unsigned long long* class_head;  // device: first request of the class with work left,
                                   // then the copies at kServeTotal and kServeStop
  int cls, cap;                 // cap: ring positions per class
  int PB, PR, PEX;
  int poll_host;                // 1: a claim that finds no device copy reads the class
                                // tail in host memory and fills the copy; 0: copies
                                // are filled by the kernel's own pollers
  unsigned long long idle_ns;   // exit after this long without work
  unsigned long long gen;       // launch generation of this kernel
};

template <class T>
__device__ __forceinline__ T volatile_load(const T* p) {
  return *const_cast<const volatile T*>(p);
}

__device__ __forceinline__ unsigned long long load_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed loads of mapped host memory that do not depend on one another are
// in flight together; a fence.acq_rel.sys after them gives them acquire
// ordering for the loads that follow (one round trip to host memory for the
// lot instead of one each).
__device__ __forceinline__ unsigned long long load_relaxed_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_sys() {
  asm volatile("fence.acq_rel.sys;" ::: "memory");
}

// True when tag a belongs to an earlier request than tag b.
__device__ __forceinline__ bool tag_older(unsigned long long a, unsigned long long b) {
  return int32_t(uint32_t(a) - uint32_t(b)) < 0;
}

// A work unit (CTA or warp, one thread calls) starts or ends serving its
// class. The unit that brings the count to zero records the generation.
__device__ __forceinline__ void serve_unit_enter(const ServeArgs& s) {
  atomicAdd_system(&s.ctrl->live[s.cls], 1);
}
__device__ __forceinline__ void serve_unit_exit(const ServeArgs& s) {
  __threadfence_system();
  if (atomicSub_system(&s.ctrl->live[s.cls], 1) == 1)
    atomicMax_system(&s.ctrl->exited_gen[s.cls], s.gen);
}

// A serving work unit: slot << 45 | class-ring position << 24 | instance
// (slots < 2^18, positions < 2^21, instances < 2^24).
__device__ __forceinline__ int64_t serve_unit(int sl, unsigned pos, unsigned long long inst) {
  return (int64_t(sl) << 45) | (int64_t(pos) << 24) | int64_t(inst);
}
__device__ __forceinline__ int unit_slot(int64_t w) { return int(w >> 45); }
__device__ __forceinline__ unsigned unit_pos(int64_t w) { return unsigned(w >> 24) & 0x1fffffu; }
__device__ __forceinline__ int unit_inst(int64_t w) { return int(w & 0xffffff); }

__device__ __forceinline__ unsigned serve_pos(const ServeArgs& s, int cls, unsigned long long head) {
  return unsigned(cls) * unsigned(s.cap) + unsigned(head % unsigned(s.cap));
}
__device__ __forceinline__ unsigned serve_pos(const ServeArgs& s, unsigned long long head) {
  return serve_pos(s, s.cls, head);
}

// 8-byte word copies (volatile: they bypass L1, whose lines could be stale
// for a position or slot reused since).
template <class T>
__device__ __forceinline__ void copy_words_volatile(T* dst, const T* src) {
  static_assert(sizeof(T) % 8 == 0, "copied in 8-byte words");
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(dst);
  constexpr int NW = int(sizeof(T) / 8);
  // every word's load first, so that they travel together (a source in
  // mapped host memory costs one round trip for the lot, not one per word)
  unsigned long long w[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) w[k] = volatile_load(a + k);
#pragma unroll
  for (int k = 0; k < NW; ++k) *const_cast<volatile unsigned long long*>(b + k) = w[k];
}

// The device copy of the request at sequence number `head` of the class, once
// that request is known to be published (head < class tail, read with
// acquire). Fills it from mapped host memory if it is missing.
__device__ __forceinline__ const ServeMirror* serve_fill_mirror(const ServeArgs& s, int cls,
                                                                unsigned long long head) {
  const unsigned pos = serve_pos(s, cls, head);
  ServeMirror* m = s.mirror + pos;
  if (volatile_load(&m->seq) == head + 1) {
    __threadfence();  // the copy's fields after its valid mark
    return m;
  }
  const ServeEntry* ep = s.class_ring + pos;
  const unsigned long long sn = volatile_load(&ep->slot_ninst);
  const unsigned long long t = volatile_load(&ep->ticket);
  copy_words_volatile(&m->d, &s.descs[int(sn >> 32)].d);
  *const_cast<volatile unsigned long long*>(&m->slot_ninst) = sn;
  *const_cast<volatile unsigned long long*>(&m->ticket) = t;
  __threadfence();  // the fields before the valid mark
  *const_cast<volatile unsigned long long*>(&m->seq) = head + 1;
  return m;
}

// The device copy of the request at sequence number `head` if it is already
// valid (then the request is published and no host memory is read), else
// nullptr.
__device__ __forceinline__ const ServeMirror* serve_valid_mirror(const ServeArgs& s,
                                                                 unsigned long long head) {
  const ServeMirror* m = s.mirror + serve_pos(s, head);
  if (volatile_load(&m->seq) != head + 1) return nullptr;
  __threadfence();
  return m;
}

// One claim attempt on the request at the class head (its device copy m).
// Returns the claimed work unit, or -1 when that request has nothing left to
// hand out (the head is then advanced past it).
__device__ __forceinline__ int64_t serve_claim_at(const ServeArgs& s, unsigned long long head,
                                                  const ServeMirror* m) {
  const unsigned pos = serve_pos(s, head);
  const unsigned long long sn = volatile_load(&m->slot_ninst);
  const unsigned long long ticket = volatile_load(&m->ticket);
  const int sl = int(sn >> 32);
  const unsigned long long n = sn & 0xffffffffull;
  const unsigned long long tag = ticket & 0xffffffffull;
  unsigned long long* cw = &s.counts[pos].claim;
  unsigned long long w = volatile_load(cw);
  while (true) {
    const unsigned long long wt = w >> 32;
    if (wt == tag) {
      if ((w & 0xffffffffull) >= n) break;  // fully handed out
      const unsigned long long old = atomicAdd(cw, 1ull);
      const unsigned long long inst = old & 0xffffffffull;
      if ((old >> 32) != tag || inst >= n) break;
      return serve_unit(sl, pos, inst);
    }
    if (!tag_older(wt, tag)) break;  // a later request holds the position: this one is done
    // first claim of this request: the word still holds an earlier one
    const unsigned long long prev = atomicCAS(cw, w, (tag << 32) | 1ull);
    if (prev == w) {
      s.comp[sl].t_first_ns = global_timer_ns();
      return serve_unit(sl, pos, 0);
    }
    w = prev;
  }
  atomicCAS(&s.class_head[s.cls], head, head + 1ull);  // request fully handed out
  return -1;
}

// One claim of the request at the head, if there is one: through its valid
// device copy, else after reading the class tail (acquire) and filling the
// copy. -1: that request is fully handed out; -2: nothing is published.
__device__ __forceinline__ int64_t serve_claim_head(const ServeArgs& s) {
  const unsigned long long head = volatile_load(&s.class_head[s.cls]);
  const ServeMirror* m = serve_valid_mirror(s, head);
  if (m == nullptr) {
    if (!s.poll_host || head >= load_acquire_sys(&s.ctrl->class_tail[s.cls])) return -2;
    m = serve_fill_mirror(s, s.cls, head);
  }
  return serve_claim_at(s, head, m);
}

// One thread finds an unclaimed instance of the oldest request of its class
// and returns it. Waits are bounded: -1 on the stop flag or after idle_ns of
// global time without work.
__device__ __forceinline__ int64_t serve_claim_wait(const ServeArgs& s) {
  const uint64_t t0 = global_timer_ns();
  while (true) {
    const int64_t w = serve_claim_head(s);
    if (w >= 0) return w;
    if (w == -1) continue;  // the head moved on: try the next request
    if (!s.poll_host) return -1;  // a class body of the warp serving kernel returns
    if (volatile_load(&s.ctrl->stop)) return -1;
    if (global_timer_ns() - t0 > s.idle_ns) return -1;
    __nanosleep(256);
  }
}

// Non-blocking claim by one thread: -2 when no work is available yet (try
// again later; the stop flag is seen by the waiting claim that follows).
__device__ __forceinline__ int64_t serve_claim_try(const ServeArgs& s) {
  while (true) {
    const int64_t w = serve_claim_head(s);
    if (w != -1) return w;
  }
}


// The descriptor of a work unit's request, from its device copy.
__device__ __forceinline__ cg_desc serve_desc(const ServeArgs& s, int64_t w) {
  cg_desc d;
  copy_words_volatile(&d, &s.mirror[unit_pos(w)].d);
  return d;
}

// Thread 0, after an instance's outputs and status are stored: counts it and,
// for the request's last instance, publishes the completion to the host.
__device__ __forceinline__ void serve_done(const ServeArgs& s, int64_t w, int status) {
  const int sl = unit_slot(w);
  const unsigned pos = unit_pos(w);
  const ServeMirror* m = s.mirror + pos;
  const unsigned long long n = volatile_load(&m->slot_ninst) & 0xffffffffull;
  const unsigned long long ticket = volatile_load(&m->ticket);
  const unsigned long long tag = ticket & 0xffffffffull;
  const unsigned long long st = (unsigned long long)(status & 0xff);
  // the instance's outputs before its count (the unit that publishes the
  // completion fences at system scope after seeing every count)
  __threadfence();
  unsigned long long* dw = &s.counts[pos].done;
  unsigned long long v = volatile_load(dw), now = 0;
  while (true) {
    if ((v >> 32) == tag) {
      // the status bits first, so that the last count sees every instance's
      if (st) atomicOr(dw, st);
      now = (atomicAdd(dw, 1ull << 8) + (1ull << 8)) | st;
      break;
    }
    // first finished instance of this request: start the count
    const unsigned long long next = (tag << 32) | (1ull << 8) | st;
    const unsigned long long prev = atomicCAS(dw, v, next);
    if (prev == v) {
      now = next;
      break;
    }
    v = prev;
  }
  if (((now >> 8) & 0xffffffull) == n) {
    __threadfence_system();
    ServeCompletion* c = s.comp + sl;
    c->status = int(now & 0xffull);
    c->t_done_ns = global_timer_ns();
    __threadfence_system();
    *const_cast<volatile unsigned long long*>(&c->seq) = ticket + 1;
  }
}

__device__ __forceinline__ DetItem det_item(const ServeArgs& s, int64_t w) {
  const cg_desc d = serve_desc(s, w);
  const int2 wu = make_int2(0, unit_inst(w));
  BatchArgs b{};
  b.desc = &d;
  b.work = &wu;
  return det_item(b, 0);
}

__device__ __forceinline__ PreItem pre_item(const ServeArgs& s, int64_t w) {
  const cg_desc d = serve_desc(s, w);
  const int2 wu = make_int2(0, unit_inst(w));
  BatchArgs b{};
  b.desc = &d;
  b.work = &wu;
  return pre_item(b, 0);
}


// Work-source hooks of the serving sources.
template <> struct SrcTraits<ServeArgs> { static constexpr bool kDyn = true; };
__device__ __forceinline__ void src_done(const ServeArgs& s, int64_t w, int status) {
  serve_done(s, w, status);
}
__device__ __forceinline__ int64_t src_count(const ServeArgs&) { return 0; }

// Lane 0 claims, every lane gets the unit (-1: none).
__device__ __forceinline__ int64_t warp_claim(const ServeArgs& s) {
  int64_t w = -1;
  if ((threadIdx.x & 31) == 0) w = serve_claim_wait(s);
  return __shfl_sync(0xffffffffu, w, 0);
}

// Claim without waiting: -2 when the class has nothing yet.
__device__ __forceinline__ int64_t warp_try(const ServeArgs& s) {
  int64_t w = -1;
  if ((threadIdx.x & 31) == 0) w = serve_claim_try(s);
  return __shfl_sync(0xffffffffu, w, 0);
}

// ---------------------------------------------------------------------------
// Serving: one kernel for the warp-per-instance classes
// ---------------------------------------------------------------------------

// Classes 0-2 detect with 8, 16, 32 padded users, 3-5 precode, 6-8 detect with
// the exact tracker (Eq. 10) with 8, 16 and 32 padded users.
constexpr int kWarpClasses = 9;
static_assert(kWarpClasses < kServeMaxClasses, "a class index past the warp classes remains");
// Every warp owns a slice large enough for any class, since the warps of one
// CTA may serve different classes at the same time.
constexpr uint32_t kServeSlice = WarpCfg<32>::WARP_BYTES;
static_assert(WarpCfg<8>::WARP_BYTES <= kServeSlice && WarpCfg<16>::WARP_BYTES <= kServeSlice &&
                  WarpCfg<32>::FRAG_BYTES <= kServeSlice,
              "serving slice must hold every class");

// Kernel parameters: the kernel's own ServeArgs (cls = its liveness counter,
// idle_ns = its idle limit) and one copy per class with cls = the class and
// idle_ns = 0, so that a class body returns once its class has no work. The
// copies live in the parameter space, which the bodies read in place.
struct ServeWarpArgs {
  ServeArgs k;
  ServeArgs c[kWarpClasses];
};

// One class body as a called function, so that each class keeps the
// register allocation it has in its own kernel.
template <int UT, int EL, bool X3>
__device__ __noinline__ void serve_detect(const ServeArgs& s, unsigned char* mine) {
  detect_warp_body<UT, EL, X3>(s, mine);
}
template <int UT, int EL, bool X3>
__device__ __noinline__ void serve_precode(const ServeArgs& s, unsigned char* mine) {
  precode_warp_body<UT, EL, X3>(s, mine);
}
template <int UT, int EL, bool X3>
__device__ __noinline__ void serve_detect_exact(const ServeArgs& s, unsigned char* mine) {
  detect_warp_body<UT, EL, X3, ServeArgs, SOLVE_CG_EXACT>(s, mine);
}

template <int EL, bool X3>
__device__ __forceinline__ void serve_class(int c, const ServeWarpArgs& p, unsigned char* mine) {
  switch (c) {
    case 0: serve_detect<8, EL, X3>(p.c[0], mine); break;
    case 1: serve_detect<16, EL, X3>(p.c[1], mine); break;
    case 2: serve_detect<32, EL, X3>(p.c[2], mine); break;
    case 3: serve_precode<8, EL, X3>(p.c[3], mine); break;
    case 4: serve_precode<16, EL, X3>(p.c[4], mine); break;
    case 5: serve_precode<32, EL, X3>(p.c[5], mine); break;
    case 6: serve_detect_exact<8, EL, X3>(p.c[6], mine); break;
    case 7: serve_detect_exact<16, EL, X3>(p.c[7], mine); break;
    default: serve_detect_exact<32, EL, X3>(p.c[8], mine); break;
  }
}

// Lane 0: the first class, starting at `home`, whose head request has its
// device copy (so it is published), or -1. Device memory only.
__device__ __forceinline__ int serve_pick(const ServeArgs& s, int home) {
  for (int j = 0; j < kWarpClasses; ++j) {
    const int c = home + j < kWarpClasses ? home + j : home + j - kWarpClasses;
    const unsigned long long head = volatile_load(&s.class_head[c]);
    if (volatile_load(&s.mirror[serve_pos(s, c, head)].seq) == head + 1) return c;
  }
  return -1;
}

// Lane 0 of an idle warp whose turn it is: reads the stop flag and the
// published-request total from mapped host memory. When the total has moved
// it fills the device copies of the new requests of every class (up to 64
// per class and call), and once none is left without one it raises the
// device copy of the total, which is what the other idle warps watch. So
// host memory sees a few reads per microsecond, not one per warp, and the
// warps' claims never read it.
__device__ __forceinline__ void serve_poll_host(const ServeArgs& s) {
  // the stop flag and the total travel together; the class tails, read
  // after the total's acquire, are at least as new as it implies and travel
  // together too; the fence then orders the entries and descriptors read
  // after them
  const int stop = volatile_load(&s.ctrl->stop);
  const unsigned long long total = load_acquire_sys(&s.ctrl->class_tail[kServeTotal]);
  if (stop) {
    *const_cast<volatile unsigned long long*>(&s.class_head[kServeStop]) = 1ull;
    return;
  }
  if (total <= volatile_load(&s.class_head[kServeTotal])) return;
  unsigned long long tails[kWarpClasses];
#pragma unroll
  for (int c = 0; c < kWarpClasses; ++c) tails[c] = load_relaxed_sys(&s.ctrl->class_tail[c]);
  fence_acq_rel_sys();
  bool all = true;
#pragma unroll
  for (int c = 0; c < kWarpClasses; ++c) {
    const unsigned long long tail = tails[c];
    const unsigned long long head = volatile_load(&s.class_head[c]);
    const unsigned long long end = tail < head + 64 ? tail : head + 64;
    if (end < tail) all = false;
    for (unsigned long long h = head; h < end; ++h) serve_fill_mirror(s, c, h);
  }
  if (!all) return;  // the next poll goes on with the rest
  __threadfence();   // the copies before the total that announces them
  atomicMax(&s.class_head[kServeTotal], total);
}

// Idle warps that read host memory in each window of 2^kPollWindowShift ns:
// 1 in kPollSlots. An idle warp sleeps at most kIdleSleepNs between looks,
// so a request published at low load waits about one window to be seen.
#ifndef CGM_POLL_SHIFT
#define CGM_POLL_SHIFT 8
#endif
#ifndef CGM_IDLE_SLEEP_NS
#define CGM_IDLE_SLEEP_NS 128
#endif
constexpr int kPollSlots = 128;
constexpr int kPollWindowShift = CGM_POLL_SHIFT;
constexpr unsigned kIdleSleepNs = CGM_IDLE_SLEEP_NS;

// Each warp serves its home class (warps are spread evenly over the classes)
// while that class has work, and otherwise the next class in turn that has
// some, so a request can use every warp of the grid when the others are
// idle. A class body returns as soon as its class has nothing left to hand
// out. Idle warps watch the device copy of the published-request total and
// look at the classes only when it has moved; a rotating few of them bring
// it up to date from host memory (serve_poll_host). Warps exit after
// idle_ns without work or on the stop flag. s.cls is the liveness counter
// of this kernel.
template <int EL, bool X3>
__global__ void __launch_bounds__(kServeThreads, 1)
    warp_serve_kernel(const __grid_constant__ ServeWarpArgs p) {
  const ServeArgs& s = p.k;
  const int lane = threadIdx.x & 31;
  unsigned char* mine = warp_slice<kServeSlice>();
  if (lane == 0) serve_unit_enter(s);
  const int gw = int(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  const int home = gw % kWarpClasses;
  unsigned long long t_idle = global_timer_ns(), seen = ~0ull;
  unsigned sleep_ns = 128;
  while (true) {
    int pick = -1;
    if (lane == 0) {
      if (volatile_load(&s.class_head[kServeStop])) {
        pick = -2;
      } else {
        const unsigned long long total = volatile_load(&s.class_head[kServeTotal]);
        if (total != seen) {
          pick = serve_pick(s, home);
          if (pick < 0) seen = total;  // nothing new until the total moves
        }
        if (pick == -1) {
          const unsigned long long now = global_timer_ns();
          if (int((now >> kPollWindowShift) % kPollSlots) == gw % kPollSlots)
            serve_poll_host(s);
          if (now - t_idle > s.idle_ns) {
            pick = -2;
          } else {
            __nanosleep(sleep_ns);
            sleep_ns = sleep_ns < kIdleSleepNs ? 2 * sleep_ns : kIdleSleepNs;
          }
        }
      }
    }
    pick = __shfl_sync(0xffffffffu, pick, 0);
    if (pick == -2) break;
    if (pick < 0) continue;
    serve_class<EL, X3>(pick, p, mine);
    t_idle = global_timer_ns();
    sleep_ns = 128;
    seen = ~0ull;
  }
  if (lane == 0) serve_unit_exit(s);
}

}  // namespace cgm
