// Serving: requests (one mixture each) arrive at any time, are admitted as device memory and
// stream slots free up, and run concurrently on the GPU (fca_server_* in fca.h).
//
// One worker thread owns the GPU side. It admits queued requests oldest first while a stream
// slot is free: the oldest when its device memory fits in the arena; when it does not, a later
// request that fits may go ahead of it, at most kMaxBypass times per waiting request (so a
// large request waiting for room does not hold up the small ones behind it, and is not
// starved by them). It enqueues the whole
// job of an admitted request on its slot's stream (host-to-device copies of the inputs, the
// one-mixture EM kernels, device-to-host copies of the outputs and of the status word, and an
// event), and polls the events of the requests in flight. When a request's event completes its
// memory and slot return to the pools and its waiter is woken, so a request arriving while
// others run is admitted as soon as room frees up and its kernels overlap theirs on the
// device. A request's results are those it gets alone: its kernels are the one-mixture ones,
// whose arithmetic does not depend on what else runs.
//
// The arena is one device allocation made at creation; requests get 256-byte aligned
// sub-blocks by first fit over an ordered free list (adjacent free blocks merge), so serving
// allocates no device memory per request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fca.h"
#include "fca_internal.h"

using namespace fca;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = up256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = up256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

// Byte offsets of one request's buffers inside its arena block.
struct ReqLayout {
  size_t status, y, v0, S0, vfloor, v, v_prev, P, P_prev, lam, lam_prev, ldet, ldet_prev, S,
      S_prev, llf, ll, PH, PinvH, lam32, x1, x2, total;
};

ReqLayout req_layout(int M, int F, int N, int iters) {
  ReqLayout L;
  const size_t f = F, fn = (size_t)F * N, fnm = fn * M, mm = (size_t)M * M;
  const size_t it = iters > 0 ? iters : 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += up256(bytes + 16);
    return at;
  };
  L.status = take(sizeof(int));
  L.y = take(fnm * 8);
  L.v0 = take(2 * fn * sizeof(double));
  L.S0 = take(2 * f * mm * 16);
  L.vfloor = take(f * 4);
  L.v = take(2 * fn * 4);
  L.v_prev = take(2 * fn * 4);
  L.P = take(f * mm * 16);
  L.P_prev = take(f * mm * 16);
  L.lam = take(f * M * 8);
  L.lam_prev = take(f * M * 8);
  L.ldet = take(f * 8);
  L.ldet_prev = take(f * 8);
  L.S = take(2 * f * mm * 16);
  L.S_prev = take(2 * f * mm * 16);
  L.llf = take(it * f * 8);
  L.ll = take(it * 8);
  L.PH = take(f * mm * 8);
  L.PinvH = take(f * mm * 8);
  L.lam32 = take(f * M * 4);
  L.x1 = take(fnm * 8);
  L.x2 = take(fnm * 8);
  L.total = o;
  return L;
}

struct Pending {
  uint64_t ticket;
  fca_request r;
  size_t bytes;
  double t_submit;
  int bypassed = 0;  // later requests admitted ahead of this one while it waited for memory
};

// Admission: at most this many later requests go ahead of a request waiting for memory, found
// among the next kBypassScan requests of the queue.
constexpr int kMaxBypass = 8;
constexpr size_t kBypassScan = 32;

struct Running {
  uint64_t ticket;
  fca_request r;
  size_t off, bytes;
  int slot;
  cudaError_t launch_error;
};

struct Info {
  bool done = false;
  fca_request_info info;
};

bool request_ok(const fca_request* r) {
  if (!r) return false;
  if (r->M < 1 || r->M > 8 || r->F < 1 || r->N < 1 || r->iters < 0) return false;
  if ((int64_t)r->F * r->N * r->M >= ((int64_t)1 << 31)) return false;
  if (r->form != FCA_FORM_FAST && r->form != FCA_FORM_CONVENTIONAL) return false;
  return r->y && r->v0 && r->S0 && r->x1 && r->x2;
}

}  // namespace

struct fca_server {
  int device = 0;
  size_t budget = 0;
  unsigned char* base = nullptr;
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  int* status_host = nullptr;  // pinned, one per slot
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::vector<Running> running;
  std::unordered_map<uint64_t, Info> infos;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::thread worker;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0;
  int max_inflight = 0;
  cudaError_t worker_error = cudaSuccess;
};

namespace {

// Enqueue the whole job of one admitted request on `st`.
cudaError_t launch_request(fca_server* s, const fca_request& r, unsigned char* blk, int slot,
                           cudaStream_t st) {
  const ReqLayout L = req_layout(r.M, r.F, r.N, r.iters);
  const int M = r.M, F = r.F, N = r.N, it = r.iters;
  const size_t fn = (size_t)F * N, fnm = fn * M, mm = (size_t)M * M;
  int* status = reinterpret_cast<int*>(blk + L.status);
  void* y = blk + L.y;
  double* v0 = reinterpret_cast<double*>(blk + L.v0);
  double2* S0 = reinterpret_cast<double2*>(blk + L.S0);
  float* vfloor = reinterpret_cast<float*>(blk + L.vfloor);
  float* v = reinterpret_cast<float*>(blk + L.v);
  float* v_prev = reinterpret_cast<float*>(blk + L.v_prev);
  double* ll = reinterpret_cast<double*>(blk + L.ll);
  float2* x1 = reinterpret_cast<float2*>(blk + L.x1);
  float2* x2 = reinterpret_cast<float2*>(blk + L.x2);
  cudaError_t e;
#define S_TRY(expr)                              \
  do {                                           \
    if ((e = (expr)) != cudaSuccess) return e;   \
  } while (0)
  S_TRY(cudaMemcpyAsync(y, r.y, fnm * 8, cudaMemcpyDefault, st));
  S_TRY(cudaMemcpyAsync(v0, r.v0, 2 * fn * sizeof(double), cudaMemcpyDefault, st));
  S_TRY(cudaMemcpyAsync(S0, r.S0, 2 * (size_t)F * mm * 16, cudaMemcpyDefault, st));
  S_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  int nk = 0;
  // FastFCA requests solve the generalised eigenproblem of S0 (Eq. (GEVD)) in the same pass.
  PrepareExtra ex;
  std::memset(&ex, 0, sizeof(ex));
  ex.max_sweeps = kDefaultSweeps;
  ex.gevd_mode = kDefaultGevdMode;
  if (r.form == FCA_FORM_FAST) {
    ex.S = S0;
    ex.P = reinterpret_cast<double2*>(blk + L.P);
    ex.lam = reinterpret_cast<double*>(blk + L.lam);
    ex.logdetS2 = reinterpret_cast<double*>(blk + L.ldet);
  }
  S_TRY(launch_prepare(M, 0, F, N, y, nullptr, v0, v, vfloor, status, st, nullptr,
                       r.form == FCA_FORM_FAST ? &ex : nullptr));
  ++nk;
  const bool res = em_resident(M, 0, N);
  const int res_bytes = res ? (int)em_dyn_smem(M, 0, N) : 0;
  double* llf = reinterpret_cast<double*>(blk + L.llf);
  if (r.form == FCA_FORM_FAST) {
    if (it > 0) {
      FastEmArgs a;
      std::memset(&a, 0, sizeof(a));
      a.F = F;
      a.N = N;
      a.iters = it;
      a.res_bytes = res_bytes;
      a.y = y;
      a.vfloor = vfloor;
      a.v_in = v;
      a.v = v;
      a.v_prev = v_prev;
      a.P = ex.P;
      a.lam = ex.lam;
      a.logdetS2 = ex.logdetS2;
      a.P_prev = reinterpret_cast<double2*>(blk + L.P_prev);
      a.lam_prev = reinterpret_cast<double*>(blk + L.lam_prev);
      a.logdetS2_prev = reinterpret_cast<double*>(blk + L.ldet_prev);
      a.llf = llf;
      a.status = status;
      a.max_sweeps = kDefaultSweeps;
      a.gevd_mode = kDefaultGevdMode;
      S_TRY(launch_fast_em(M, 0, a, st));
      ++nk;
    }
    ParamArgs sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.F = F;
    sp.status = status;
    sp.P = it > 0 ? reinterpret_cast<double2*>(blk + L.P_prev) : ex.P;
    sp.lam = it > 0 ? reinterpret_cast<double*>(blk + L.lam_prev) : ex.lam;
    sp.PH = reinterpret_cast<float2*>(blk + L.PH);
    sp.PinvH = reinterpret_cast<float2*>(blk + L.PinvH);
    sp.lam32 = reinterpret_cast<float*>(blk + L.lam32);
    S_TRY(launch_sep_prep(M, sp, st));
    ++nk;
    SepFastArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.F = F;
    sa.N = N;
    sa.y = y;
    sa.v = it > 0 ? v_prev : v;
    sa.PH = sp.PH;
    sa.PinvH = sp.PinvH;
    sa.lam = sp.lam32;
    sa.x1 = x1;
    sa.x2 = x2;
    S_TRY(launch_sep_fast(M, 0, sa, st));
    ++nk;
  } else {
    double2* S = reinterpret_cast<double2*>(blk + L.S);
    double2* S_prev = reinterpret_cast<double2*>(blk + L.S_prev);
    if (it > 0) {
      ConvEmArgs a;
      std::memset(&a, 0, sizeof(a));
      a.F = F;
      a.N = N;
      a.iters = it;
      a.res_bytes = res_bytes;
      a.y = y;
      a.vfloor = vfloor;
      a.v_in = v;
      a.v = v;
      a.v_prev = v_prev;
      S_TRY(cudaMemcpyAsync(S, S0, 2 * (size_t)F * mm * 16, cudaMemcpyDeviceToDevice, st));
      a.S_in = S;
      a.S = S;
      a.S_prev = S_prev;
      a.llf = llf;
      a.status = status;
      S_TRY(launch_conv_em(M, 0, a, st));
      ++nk;
    }
    SepConvArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.F = F;
    sa.N = N;
    sa.y = y;
    sa.v = it > 0 ? v_prev : v;
    sa.S = it > 0 ? S_prev : S0;
    sa.x1 = x1;
    sa.x2 = x2;
    sa.status = status;
    S_TRY(launch_sep_conv(M, 0, sa, st));
    ++nk;
  }
  if (it > 0) {
    S_TRY(launch_ll_reduce(F, it, llf, ll, st));
    ++nk;
    if (r.loglik) S_TRY(cudaMemcpyAsync(r.loglik, ll, (size_t)it * 8, cudaMemcpyDefault, st));
  }
  if (r.v) S_TRY(cudaMemcpyAsync(r.v, v, 2 * fn * sizeof(float), cudaMemcpyDefault, st));
  S_TRY(cudaMemcpyAsync(r.x1, x1, fnm * 8, cudaMemcpyDefault, st));
  S_TRY(cudaMemcpyAsync(r.x2, x2, fnm * 8, cudaMemcpyDefault, st));
  S_TRY(cudaMemcpyAsync(&s->status_host[slot], status, sizeof(int), cudaMemcpyDeviceToHost, st));
  S_TRY(cudaEventRecord(s->events[slot], st));
  note_launches(nk);
#undef S_TRY
  return cudaSuccess;
}

void worker_main(fca_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // Admit the oldest request while it fits; while it does not, a later one that fits may go
    // ahead of it (bounded by kMaxBypass).
    while (!s->queue.empty() && !s->free_slots.empty()) {
      size_t off = 0, pick = 0;
      if (!s->arena.alloc(s->queue.front().bytes, &off)) {
        if (s->queue.front().bypassed >= kMaxBypass) break;
        pick = s->queue.size();
        for (size_t i = 1; i < s->queue.size() && i <= kBypassScan; ++i) {
          if (s->arena.alloc(s->queue[i].bytes, &off)) {
            pick = i;
            break;
          }
        }
        if (pick == s->queue.size()) break;
        ++s->queue.front().bypassed;
      }
      const Pending p = s->queue[pick];
      Running run;
      run.ticket = p.ticket;
      run.r = p.r;
      run.off = off;
      run.bytes = p.bytes;
      run.slot = s->free_slots.back();
      s->free_slots.pop_back();
      s->infos[p.ticket].info.t_admit = now_s();
      s->queue.erase(s->queue.begin() + (ptrdiff_t)pick);
      lk.unlock();
      run.launch_error = launch_request(s, run.r, s->base + off, run.slot, s->streams[run.slot]);
      lk.lock();
      s->running.push_back(run);
      s->max_inflight = std::max(s->max_inflight, (int)s->running.size());
    }
    // Retire completed requests.
    bool progressed = false;
    for (size_t i = 0; i < s->running.size();) {
      Running& run = s->running[i];
      cudaError_t q = cudaSuccess;
      if (run.launch_error == cudaSuccess) {
        q = cudaEventQuery(s->events[run.slot]);
        if (q == cudaErrorNotReady) {
          ++i;
          continue;
        }
      }
      if (run.launch_error != cudaSuccess) {
        // Whatever was enqueued before the failure must finish before the memory is reused.
        cudaStreamSynchronize(s->streams[run.slot]);
        cudaGetLastError();
      }
      Info& inf = s->infos[run.ticket];
      fca_status st = FCA_OK;
      if (run.launch_error != cudaSuccess || q != cudaSuccess) {
        st = FCA_ERR_CUDA;
        if (run.launch_error == cudaSuccess) s->worker_error = q;
      } else if (s->status_host[run.slot] != 0) {
        st = (fca_status)s->status_host[run.slot];
      }
      inf.info.status = st;
      inf.info.t_done = now_s();
      inf.done = true;
      if (st == FCA_OK) ++s->completed;
      else ++s->failed;
      s->arena.release(run.off, run.bytes);
      s->free_slots.push_back(run.slot);
      s->running[i] = s->running.back();
      s->running.pop_back();
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    if (s->stopping && s->queue.empty() && s->running.empty()) break;
    if (s->running.empty()) {
      s->cv_work.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
    } else if (!progressed) {
      // Requests are in flight: poll their events again shortly (a submission wakes us now).
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

extern "C" {

fca_status fca_server_create(const fca_server_config* cfg, fca_server** out) {
  if (!out) return FCA_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->device_bytes < 4096 || cfg->max_inflight < 1 || cfg->max_inflight > 64)
    return FCA_ERR_ARG;
  fca_server* s = new (std::nothrow) fca_server;
  if (!s) return FCA_ERR_NOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return FCA_ERR_CUDA;
  }
  s->budget = (size_t)cfg->device_bytes & ~(size_t)255;
  cudaError_t e = cudaMalloc((void**)&s->base, s->budget);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->status_host, cfg->max_inflight * sizeof(int), 0);
  for (int i = 0; i < cfg->max_inflight && e == cudaSuccess; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    s->streams.push_back(st);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    s->events.push_back(ev);
    s->free_slots.push_back(cfg->max_inflight - 1 - i);
  }
  if (e != cudaSuccess) {
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    if (s->status_host) cudaFreeHost(s->status_host);
    if (s->base) cudaFree(s->base);
    cudaGetLastError();
    delete s;
    return e == cudaErrorMemoryAllocation ? FCA_ERR_NOMEM : FCA_ERR_CUDA;
  }
  s->arena.reset(s->budget);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return FCA_OK;
}

size_t fca_server_request_bytes(int32_t M, int32_t F, int32_t N, int32_t iters) {
  if (M < 1 || M > 8 || F < 1 || N < 1 || iters < 0) return 0;
  return req_layout(M, F, N, iters).total;
}

fca_status fca_server_submit(fca_server* s, const fca_request* r, uint64_t* ticket) {
  if (!s || !ticket || !request_ok(r)) return FCA_ERR_ARG;
  const size_t bytes = req_layout(r->M, r->F, r->N, r->iters).total;
  if (bytes > s->budget) return FCA_ERR_NOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return FCA_ERR_STATE;
  Pending p;
  p.ticket = s->next_ticket++;
  p.r = *r;
  p.bytes = bytes;
  p.t_submit = now_s();
  Info& inf = s->infos[p.ticket];
  std::memset(&inf.info, 0, sizeof(inf.info));
  inf.info.t_submit = p.t_submit;
  s->queue.push_back(p);
  ++s->submitted;
  *ticket = p.ticket;
  s->cv_work.notify_one();
  return FCA_OK;
}

fca_status fca_server_wait(fca_server* s, uint64_t ticket, int64_t timeout_ms, fca_request_info* info) {
  if (!s) return FCA_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->infos.find(ticket);
  if (it == s->infos.end()) return FCA_ERR_ARG;
  auto ready = [&] { return s->infos[ticket].done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return FCA_ERR_TIMEOUT;
  }
  const fca_request_info inf = s->infos[ticket].info;
  s->infos.erase(ticket);
  if (info) *info = inf;
  return inf.status;
}

fca_status fca_server_stats(fca_server* s, fca_server_counters* out) {
  if (!s || !out) return FCA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = s->queue.size();
  out->in_flight = s->running.size();
  out->max_in_flight = s->max_inflight;
  out->bytes_in_use = s->arena.used();
  out->bytes_peak = s->arena.peak();
  out->bytes_budget = s->budget;
  return s->worker_error == cudaSuccess ? FCA_OK : FCA_ERR_CUDA;
}

void fca_server_destroy(fca_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int old = -1;
  cudaGetDevice(&old);
  if (old != s->device) cudaSetDevice(s->device);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  if (s->status_host) cudaFreeHost(s->status_host);
  if (s->base) cudaFree(s->base);
  if (old >= 0 && old != s->device) cudaSetDevice(old);
  delete s;
}

}  // extern "C"
