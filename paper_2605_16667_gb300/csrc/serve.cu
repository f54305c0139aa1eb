// The served form: continuous batching of DialSort requests on one GPU.
//
// A server owns an HBM arena (allocated once, at creation), a ring of request
// slots in device memory, completion records in host-mapped memory, and a
// scheduler thread.  Clients submit requests that reference device-resident
// keys; the scheduler admits them in arrival order whenever a slot is free
// and the arena can hold the request's H, output and scan scratch (the HBM
// budget).  Admission writes the slot's description by DMA on a copy stream
// and publishes its first phase last.  The persistent engine kernel
// (engine.cu, served mode) picks admitted requests up while it runs, so a
// request that arrives while others are on the GPU starts as soon as a slot
// and memory free up, and its work items interleave with theirs.  Finished
// requests are reported through the mapped completion records; their H and
// output stay in the arena until the client releases them.
//
// The engine kernel leaves when it has been idle for idle_timeout_ns (every
// device wait is bounded); the scheduler relaunches it when work arrives.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace dialsort {
namespace {

uint64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

// First-fit allocator over one device region, 256-byte granules, coalescing frees.
class Arena {
 public:
  void init(char* base, size_t bytes) {
    base_ = base;
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  char* alloc(size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_[off] = bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(char* p) {
    if (!p) return;
    const size_t off = (size_t)(p - base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t size = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + size == next->first) {
      size += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += size;
        return;
      }
    }
    free_[off] = size;
  }

 private:
  char* base_ = nullptr;
  std::map<size_t, size_t> free_;  // offset -> size
  std::unordered_map<size_t, size_t> used_;
};

enum TicketState : int { T_PENDING = 0, T_ADMITTED = 1, T_DONE = 2 };

struct Ticket {
  dialsort_request_t req{};
  int state = T_PENDING;
  int slot = -1;
  char* block = nullptr;  // arena block: H | out | scratch
  uint32_t* H = nullptr;
  void* out = nullptr;
  uint64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
  uint32_t status = DIALSORT_OK;
};

}  // namespace
}  // namespace dialsort

using namespace dialsort;
using namespace dialsort::eng;

struct dialsort_server_s {
  dialsort_server_cfg_t cfg{};
  int device = -1;
  const DeviceInfo* dev = nullptr;
  uint32_t slots = 0;
  char* arena_base = nullptr;
  Arena arena;
  Req* d_reqs = nullptr;
  State* d_states = nullptr;
  Completion* h_comp = nullptr;  // mapped
  Completion* d_comp = nullptr;
  HostCtl* h_ctl = nullptr;      // mapped
  HostCtl* d_ctl = nullptr;
  Req* h_req_stage = nullptr;    // pinned, one per slot
  State* h_state_stage = nullptr;
  unsigned long long* h_word_stage = nullptr;
  unsigned long long* h_bell_stage = nullptr;  // per slot: the doorbell value its admission wrote
  unsigned long long bells = 0;
  Ctl* d_ctl_dev = nullptr;
  cudaStream_t engine_stream = nullptr, copy_stream = nullptr;
  cudaEvent_t engine_done = nullptr;
  bool engine_launched = false;
  uint32_t grid = 0;

  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Ticket> tickets;
  std::vector<int64_t> slot_ticket;   // -1 free
  std::vector<uint64_t> slot_seq;
  uint64_t next_ticket = 1, next_seq = 0;
  uint32_t busy_slots = 0;
  std::atomic<bool> quit{false};
  std::thread worker;
  dialsort_status_t fatal = DIALSORT_OK;

  size_t block_bytes(const dialsort_request_t& r, Req* plan) const {
    ReqPlanInput in{r.keys, reinterpret_cast<uint32_t*>(256), r.kind ? reinterpret_cast<void*>(256) : nullptr, r.n,
                    r.U, r.key_bytes, r.skew <= 3 ? r.skew : 0u, 0u, true};
    (void)plan_request(in, plan);  // automatic: always applies
    size_t b = align_up((size_t)r.U * 4, 256);
    if (r.kind) b += align_up((size_t)r.n * r.key_bytes, 256);
    return b + request_scratch_bytes(*plan);
  }

  // admit the ticket into slot s (lock held); returns false if the arena is full
  bool admit(uint64_t id, Ticket& t, uint32_t s) {
    Req plan;
    const size_t bytes = block_bytes(t.req, &plan);
    char* block = arena.alloc(bytes);
    if (!block) return false;
    t.block = block;
    t.H = reinterpret_cast<uint32_t*>(block);
    char* p = block + align_up((size_t)t.req.U * 4, 256);
    t.out = nullptr;
    if (t.req.kind) {
      t.out = p;
      p += align_up((size_t)t.req.n * t.req.key_bytes, 256);
    }
    ReqPlanInput in{t.req.keys, t.H, t.out, t.req.n, t.req.U, t.req.key_bytes, t.req.skew <= 3 ? t.req.skew : 0u,
                    0u, true};
    Req& r = h_req_stage[s];
    (void)plan_request(in, &r);
    place_request_scratch(&r, p);
    const uint64_t seq = next_seq++;
    State& st = h_state_stage[s];
    std::memset(&st, 0, sizeof(State));
    st.seq = seq;
    st.word = pack_word(seq, PH_FREE, 0);
    h_word_stage[s] = pack_word(seq, r.first_phase, 0);
    // slot description, reset state (phase FREE: nothing claimable), then the
    // state word with the first phase, last.  Only DMA: a kernel (even a
    // memset) could not start while the engine occupies every SM; the
    // request's zero phase clears its look-back descriptors on the device.
    cudaError_t e = cudaMemcpyAsync(&d_reqs[s], &r, sizeof(Req), cudaMemcpyHostToDevice, copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&d_states[s], &st, sizeof(State), cudaMemcpyHostToDevice, copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&d_states[s].word, &h_word_stage[s], 8, cudaMemcpyHostToDevice, copy_stream);
    // then the doorbell (from this slot's own staging word, which stays put until the slot is reused):
    // idle engine CTAs watch this one word and scan the ring when it changes
    h_bell_stage[s] = ++bells;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&d_ctl_dev->bell, &h_bell_stage[s], 8, cudaMemcpyHostToDevice, copy_stream);
    if (e != cudaSuccess) {
      arena.release(block);
      fatal = DIALSORT_ERR_CUDA;
      return false;
    }
    h_comp[s].seq_done = 0;
    t.state = T_ADMITTED;
    t.slot = (int)s;
    t.admit_ns = now_ns();
    slot_ticket[s] = (int64_t)id;
    slot_seq[s] = seq;
    ++busy_slots;
    return true;
  }

  void ensure_engine() {
    if (engine_launched && cudaEventQuery(engine_done) == cudaErrorNotReady) return;
    // the copy stream's admissions must be in place before the engine looks
    cudaStreamSynchronize(copy_stream);
    Launch L{};
    L.reqs = d_reqs;
    L.st = d_states;
    L.ctl = d_ctl_dev;
    L.comp = d_comp;
    L.host = d_ctl;
    L.err = dev->err;
    L.count = slots;
    L.served = 1;
    L.idle_ns = cfg.idle_timeout_ns;
    if (launch_engine(L, grid, engine_stream) != cudaSuccess ||
        cudaEventRecord(engine_done, engine_stream) != cudaSuccess) {
      fatal = DIALSORT_ERR_CUDA;
      return;
    }
    engine_launched = true;
  }

  void loop() {
    cudaSetDevice(device);
    while (!quit.load()) {
      bool active;
      {
        std::unique_lock<std::mutex> lk(mu);
        // completions
        for (uint32_t s = 0; s < slots; ++s) {
          if (slot_ticket[s] < 0) continue;
          if (h_comp[s].seq_done != slot_seq[s] + 1) continue;
          auto it = tickets.find((uint64_t)slot_ticket[s]);
          if (it != tickets.end()) {
            Ticket& t = it->second;
            t.done_ns = now_ns();
            const uint32_t err = h_comp[s].err;
            t.status = (err & ERRBIT_TIMEOUT)    ? DIALSORT_ERR_TIMEOUT
                       : (err & ERRBIT_OVERFLOW) ? DIALSORT_ERR_OVERFLOW
                       : (err & ERRBIT_KEY_RANGE) ? DIALSORT_ERR_KEY_RANGE
                                                  : DIALSORT_OK;
            t.state = T_DONE;
            t.slot = -1;
          }
          slot_ticket[s] = -1;
          --busy_slots;
          cv_done.notify_all();
        }
        // admissions, in arrival order
        while (!pending.empty() && busy_slots < slots && fatal == DIALSORT_OK) {
          const uint64_t id = pending.front();
          auto it = tickets.find(id);
          if (it == tickets.end()) {
            pending.pop_front();
            continue;
          }
          uint32_t s = 0;
          while (s < slots && slot_ticket[s] >= 0) ++s;
          if (!admit(id, it->second, s)) break;  // wait for memory to free up
          pending.pop_front();
        }
        active = busy_slots > 0;
        if (active) ensure_engine();
        if (!active && pending.empty()) {
          cv_submit.wait_for(lk, std::chrono::microseconds(200));
          continue;
        }
      }
      // requests in flight: poll completions at a short interval
      std::this_thread::yield();
    }
  }
};

namespace {

void destroy_server(dialsort_server_s* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    s->quit.store(true);
    s->cv_submit.notify_all();
    s->worker.join();
  }
  if (s->h_ctl) s->h_ctl->stop = 1;
  if (s->engine_stream) cudaStreamSynchronize(s->engine_stream);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  if (s->engine_done) cudaEventDestroy(s->engine_done);
  if (s->engine_stream) cudaStreamDestroy(s->engine_stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->d_reqs) cudaFree(s->d_reqs);
  if (s->d_states) cudaFree(s->d_states);
  if (s->h_comp) cudaFreeHost(s->h_comp);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
  if (s->h_req_stage) cudaFreeHost(s->h_req_stage);
  if (s->h_state_stage) cudaFreeHost(s->h_state_stage);
  if (s->h_word_stage) cudaFreeHost(s->h_word_stage);
  if (s->h_bell_stage) cudaFreeHost(s->h_bell_stage);
  if (s->d_ctl_dev) cudaFree(s->d_ctl_dev);
  delete s;
}

dialsort_status_t check_request(const dialsort_request_t* r) {
  if (r == nullptr || (r->key_bytes != 4 && r->key_bytes != 2) || r->U == 0 || r->n >= (1ull << 32) || r->kind > 1)
    return DIALSORT_ERR_INVALID_ARG;
  if (r->key_bytes == 2 && r->U > 65536u) return DIALSORT_ERR_INVALID_ARG;
  if (r->n > 0 && (r->keys == nullptr || (reinterpret_cast<uintptr_t>(r->keys) % r->key_bytes) != 0))
    return DIALSORT_ERR_INVALID_ARG;
  return DIALSORT_OK;
}

void fill_result(const Ticket& t, dialsort_result_t* res) {
  res->H = t.H;
  res->out = t.out;
  res->submit_ns = t.submit_ns;
  res->admit_ns = t.admit_ns;
  res->done_ns = t.done_ns;
  res->status = t.status;
}

}  // namespace

extern "C" {

dialsort_status_t dialsort_server_create(const dialsort_server_cfg_t* cfg, dialsort_server_t** out) {
  if (cfg == nullptr || out == nullptr || cfg->max_slots == 0 || cfg->max_slots > kWindow ||
      cfg->hbm_budget_bytes < 4096)
    return DIALSORT_ERR_INVALID_ARG;
  *out = nullptr;
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  dialsort_server_s* s = new (std::nothrow) dialsort_server_s();
  if (!s) return DIALSORT_ERR_INVALID_ARG;
  s->cfg = *cfg;
  if (s->cfg.idle_timeout_ns == 0) s->cfg.idle_timeout_ns = 20000000ull;  // 20 ms
  s->device = dev->device;
  s->dev = dev;
  s->slots = cfg->max_slots;
  s->slot_ticket.assign(s->slots, -1);
  s->slot_seq.assign(s->slots, 0);
  bool ok = cudaMalloc(&s->arena_base, cfg->hbm_budget_bytes) == cudaSuccess &&
            cudaMalloc(&s->d_reqs, sizeof(Req) * s->slots) == cudaSuccess &&
            cudaMalloc(&s->d_states, sizeof(State) * s->slots) == cudaSuccess &&
            cudaHostAlloc(&s->h_comp, sizeof(Completion) * s->slots, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc(&s->h_ctl, sizeof(HostCtl), cudaHostAllocMapped) == cudaSuccess &&
            cudaMallocHost(&s->h_req_stage, sizeof(Req) * s->slots) == cudaSuccess &&
            cudaMallocHost(&s->h_state_stage, sizeof(State) * s->slots) == cudaSuccess &&
            cudaMallocHost(&s->h_word_stage, sizeof(unsigned long long) * s->slots) == cudaSuccess &&
            cudaMallocHost(&s->h_bell_stage, sizeof(unsigned long long) * s->slots) == cudaSuccess &&
            cudaMalloc(&s->d_ctl_dev, sizeof(Ctl)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->engine_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->engine_done, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    std::memset(s->h_comp, 0, sizeof(Completion) * s->slots);
    std::memset(s->h_ctl, 0, sizeof(HostCtl));
    ok = cudaHostGetDevicePointer((void**)&s->d_comp, s->h_comp, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&s->d_ctl, s->h_ctl, 0) == cudaSuccess &&
         cudaMemset(s->d_states, 0, sizeof(State) * s->slots) == cudaSuccess &&
         cudaMemset(s->d_ctl_dev, 0, sizeof(Ctl)) == cudaSuccess;
  }
  if (!ok) {
    destroy_server(s);
    return DIALSORT_ERR_CUDA;
  }
  s->arena.init(s->arena_base, cfg->hbm_budget_bytes);
  s->grid = engine_grid(*dev);
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return DIALSORT_OK;
}

dialsort_status_t dialsort_server_submit(dialsort_server_t* s, const dialsort_request_t* req, uint64_t* ticket) {
  if (s == nullptr || ticket == nullptr) return DIALSORT_ERR_INVALID_ARG;
  dialsort_status_t st = check_request(req);
  if (st != DIALSORT_OK) return st;
  Req plan;
  if (s->block_bytes(*req, &plan) > s->cfg.hbm_budget_bytes) return DIALSORT_ERR_BUDGET;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != DIALSORT_OK) return s->fatal;
  const uint64_t id = s->next_ticket++;
  Ticket& t = s->tickets[id];
  t.req = *req;
  t.submit_ns = now_ns();
  s->pending.push_back(id);
  *ticket = id;
  s->cv_submit.notify_one();
  return DIALSORT_OK;
}

dialsort_status_t dialsort_server_poll(dialsort_server_t* s, uint64_t ticket, dialsort_result_t* res) {
  if (s == nullptr || res == nullptr) return DIALSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return DIALSORT_ERR_INVALID_ARG;
  if (it->second.state != T_DONE) return s->fatal != DIALSORT_OK ? s->fatal : DIALSORT_ERR_BUSY;
  fill_result(it->second, res);
  return DIALSORT_OK;
}

dialsort_status_t dialsort_server_wait(dialsort_server_t* s, uint64_t ticket, uint64_t timeout_ns,
                                       dialsort_result_t* res) {
  if (s == nullptr || res == nullptr) return DIALSORT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
  for (;;) {
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return DIALSORT_ERR_INVALID_ARG;
    if (it->second.state == T_DONE) {
      fill_result(it->second, res);
      return DIALSORT_OK;
    }
    if (s->fatal != DIALSORT_OK) return s->fatal;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto again = s->tickets.find(ticket);
      if (again != s->tickets.end() && again->second.state == T_DONE) {
        fill_result(again->second, res);
        return DIALSORT_OK;
      }
      return DIALSORT_ERR_BUSY;
    }
  }
}

dialsort_status_t dialsort_server_release(dialsort_server_t* s, uint64_t ticket) {
  if (s == nullptr) return DIALSORT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return DIALSORT_ERR_INVALID_ARG;
  if (it->second.state == T_ADMITTED) return DIALSORT_ERR_BUSY;
  if (it->second.state == T_PENDING) {
    s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), ticket), s->pending.end());
  }
  s->arena.release(it->second.block);
  s->tickets.erase(it);
  s->cv_submit.notify_one();
  return DIALSORT_OK;
}

dialsort_status_t dialsort_server_destroy(dialsort_server_t* s) {
  if (s == nullptr) return DIALSORT_ERR_INVALID_ARG;
  destroy_server(s);
  return DIALSORT_OK;
}

// ---------------------------------------------------------------- trace replay

dialsort_status_t dialsort_replay(const dialsort_trace_entry_t* trace, uint32_t count, int use_server,
                                  const dialsort_server_cfg_t* cfg, dialsort_trace_result_t* results,
                                  uint64_t* wall_ns) {
  if ((count > 0 && (trace == nullptr || results == nullptr)) || cfg == nullptr) return DIALSORT_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < count; ++i) {
    dialsort_request_t r{trace[i].keys, trace[i].n, trace[i].U, trace[i].key_bytes, trace[i].kind, 0};
    dialsort_status_t st = check_request(&r);
    if (st != DIALSORT_OK) return st;
  }
  const uint64_t t0 = now_ns() + 1000000ull;  // arrivals are offsets from 1 ms after the call
  if (use_server) {
    dialsort_server_t* srv = nullptr;
    dialsort_status_t st = dialsort_server_create(cfg, &srv);
    if (st != DIALSORT_OK) return st;
    std::vector<uint64_t> tickets(count);
    std::deque<uint32_t> open;
    auto reap = [&](bool block) {
      while (!open.empty()) {
        dialsort_result_t res;
        const uint32_t i = open.front();
        dialsort_status_t p = block ? dialsort_server_wait(srv, tickets[i], 10000000000ull, &res)
                                    : dialsort_server_poll(srv, tickets[i], &res);
        if (p == DIALSORT_ERR_BUSY && !block) {
          // later requests may have finished first: look past the head
          bool any = false;
          for (size_t k = 1; k < open.size(); ++k) {
            const uint32_t j = open[k];
            if (dialsort_server_poll(srv, tickets[j], &res) == DIALSORT_OK) {
              results[j].arrival_ns = trace[j].arrival_ns;
              results[j].done_ns = res.done_ns - t0;
              results[j].status = res.status;
              dialsort_server_release(srv, tickets[j]);
              open.erase(open.begin() + (long)k);
              any = true;
              break;
            }
          }
          if (!any) return;
          continue;
        }
        if (p != DIALSORT_OK) {
          results[i].status = p;
          results[i].done_ns = now_ns() - t0;
        } else {
          results[i].status = res.status;
          results[i].done_ns = res.done_ns - t0;
        }
        results[i].arrival_ns = trace[i].arrival_ns;
        dialsort_server_release(srv, tickets[i]);
        open.pop_front();
      }
    };
    for (uint32_t i = 0; i < count; ++i) {
      while (now_ns() < t0 + trace[i].arrival_ns) reap(false);
      dialsort_request_t r{trace[i].keys, trace[i].n, trace[i].U, trace[i].key_bytes, trace[i].kind, 0};
      if (dialsort_server_submit(srv, &r, &tickets[i]) != DIALSORT_OK) {
        dialsort_server_destroy(srv);
        return DIALSORT_ERR_INVALID_ARG;
      }
      open.push_back(i);
    }
    reap(true);
    if (wall_ns) *wall_ns = now_ns() - t0;
    return dialsort_server_destroy(srv);
  }

  // per-request plain launches: one stream, each request's kernels launched at its arrival
  const DeviceInfo* dev = device_info();
  if (!dev) return DIALSORT_ERR_CUDA;
  char* base = nullptr;
  cudaStream_t stream = nullptr;
  if (cudaMalloc(&base, cfg->hbm_budget_bytes) != cudaSuccess) return DIALSORT_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(base);
    return DIALSORT_ERR_CUDA;
  }
  Arena arena;
  arena.init(base, cfg->hbm_budget_bytes);
  struct InFlight {
    uint32_t i;
    char* block;
    cudaEvent_t ev;
  };
  std::deque<InFlight> flight;
  dialsort_status_t result = DIALSORT_OK;
  auto reap = [&](bool block) {
    while (!flight.empty()) {
      InFlight& f = flight.front();
      cudaError_t q = cudaEventQuery(f.ev);
      if (q == cudaErrorNotReady) {
        if (!block) return;
        continue;
      }
      results[f.i].arrival_ns = trace[f.i].arrival_ns;
      results[f.i].done_ns = now_ns() - t0;
      results[f.i].status = q == cudaSuccess ? DIALSORT_OK : DIALSORT_ERR_CUDA;
      arena.release(f.block);
      cudaEventDestroy(f.ev);
      flight.pop_front();
    }
  };
  for (uint32_t i = 0; i < count && result == DIALSORT_OK; ++i) {
    while (now_ns() < t0 + trace[i].arrival_ns) reap(false);
    const dialsort_trace_entry_t& e = trace[i];
    const size_t hb = align_up((size_t)e.U * 4, 256);
    const size_t ob = e.kind ? align_up((size_t)e.n * e.key_bytes, 256) : 0;
    const size_t wb = e.kind ? dialsort_reconstruct_workspace_size(e.U, e.n) : 0;
    char* block = nullptr;
    for (;;) {  // wait for memory like the server does
      block = arena.alloc(hb + ob + wb);
      if (block || flight.empty()) break;
      reap(false);
    }
    if (!block) {
      result = DIALSORT_ERR_BUDGET;
      break;
    }
    dialsort_status_t st;
    uint32_t* H = reinterpret_cast<uint32_t*>(block);
    if (e.kind == 0) {
      st = e.key_bytes == 4 ? dialsort_histogram(static_cast<const uint32_t*>(e.keys), e.n, e.U, H, stream)
                            : dialsort_histogram_u16(static_cast<const uint16_t*>(e.keys), e.n, e.U, H, stream);
    } else {
      st = e.key_bytes == 4 ? dialsort_histogram(static_cast<const uint32_t*>(e.keys), e.n, e.U, H, stream)
                            : dialsort_histogram_u16(static_cast<const uint16_t*>(e.keys), e.n, e.U, H, stream);
      if (st == DIALSORT_OK)
        st = e.key_bytes == 4
                 ? dialsort_reconstruct(H, e.U, reinterpret_cast<uint32_t*>(block + hb), e.n, block + hb + ob, wb, stream)
                 : dialsort_reconstruct_u16(H, e.U, reinterpret_cast<uint16_t*>(block + hb), e.n, block + hb + ob, wb,
                                            stream);
    }
    cudaEvent_t ev;
    if (st != DIALSORT_OK || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, stream) != cudaSuccess) {
      arena.release(block);
      result = st != DIALSORT_OK ? st : DIALSORT_ERR_CUDA;
      break;
    }
    flight.push_back({i, block, ev});
  }
  reap(true);
  if (wall_ns) *wall_ns = now_ns() - t0;
  cudaStreamDestroy(stream);
  cudaFree(base);
  return result;
}

}  // extern "C"
