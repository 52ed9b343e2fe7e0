// Batches of mixtures of uneven channel count M and length N in one job (fca_batch_* in
// fca.h).
//
// Every frequency bin of every mixture is an independent EM problem (Eq. (like) factorises
// over bins and mixtures), so a batch is a set of bins. Bins are grouped into classes by M
// (the kernels are specialised on M); inside a class the per-bin parameters (S, P, Lambda,
// log det S2, the positivity floor and the per-iteration log-likelihood) are stored in the
// one-mixture [F] layouts with F = the class's bin count, and a descriptor per bin locates its
// time-frequency points and source powers. The fused EM kernel of each class runs one CTA per
// bin over a descriptor table sorted longest bin first (the block scheduler then hands out
// the long bins first: longest-processing-time order). The classes run on their own streams,
// forked from and joined back into the caller's stream, so their kernels overlap; the whole
// job can be captured once into a CUDA graph and replayed with a single launch.
//
// Layouts (dense packing in the caller's order): mixture k's y, x1, x2 start at element
// sum_{k'<k} F N M, its v0 / v at sum 2 F N, its S0 at sum 2 F M^2. The library's own copy
// of y starts every mixture on a 16-byte boundary (vector loads).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "fca.h"
#include "fca_internal.h"

using namespace fca;

namespace {

struct BatchClass {
  int M = 0;
  int nbins = 0, Nmax = 0;
  std::vector<int> mix;            // global indices of the class's mixtures
  std::vector<int> b0;             // first class bin of each of them
  std::vector<BinDesc> host_bins;  // longest first
  BinDesc* bins = nullptr;         // device copy of host_bins
  BinDesc* sample = nullptr;       // tuning sample (device)
  int nsample = 0;
  int* mix_b0 = nullptr;
  int* mix_nb = nullptr;
  int* mix_id = nullptr;
  float* vfloor = nullptr;
  double2* S0 = nullptr;
  double2* S = nullptr;
  double2* S_prev = nullptr;
  double2* P = nullptr;
  double* lam = nullptr;
  double* ldet = nullptr;
  double2* P_prev = nullptr;
  double* lam_prev = nullptr;
  double* ldet_prev = nullptr;
  float2* sep_PH = nullptr;
  float2* sep_PinvH = nullptr;
  float* sep_lam = nullptr;
  double* llf = nullptr;
  int llf_cap = 0;
  int threads = 128;   // FastFCA launch shape
  int res_bytes = 0;
  int tuned = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

struct GraphKey {
  int form = -1, iters = -1;
  const void *ll = nullptr, *x1 = nullptr, *x2 = nullptr, *v = nullptr;
  bool operator==(const GraphKey& o) const {
    return form == o.form && iters == o.iters && ll == o.ll && x1 == o.x1 && x2 == o.x2 && v == o.v;
  }
};

fca_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FCA_OK;
  if (e == cudaErrorMemoryAllocation) return FCA_ERR_NOMEM;
  return FCA_ERR_CUDA;
}

#define B_CHECK(expr)                                 \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_status(e_);    \
  } while (0)

template <typename T>
cudaError_t balloc(T** p, size_t count) {
  *p = nullptr;
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

bool on_device(const void* ptr, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

struct DeviceGuard {
  int old = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DeviceGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

// Largest em_bin_smem of the class's bins that fits under `cap` (0 if none does).
int resident_bytes(const BatchClass& c, size_t cap) {
  size_t best = 0;
  for (const BinDesc& d : c.host_bins) {
    const size_t need = em_bin_smem(c.M, 0, d.N);
    if (need <= cap && need > best) best = need;
  }
  return (int)best;
}

}  // namespace

struct fca_batch {
  int count = 0, device = 0;
  std::vector<int> M, F, N;
  std::vector<long long> y_off, x_off, v_off, S_off;
  long long y_elems = 0, x_elems = 0, v_elems = 0, S_elems = 0;
  void* y = nullptr;
  float* v0f = nullptr;
  float* v = nullptr;
  float* v_prev = nullptr;
  int* status = nullptr;
  std::vector<BatchClass> cls;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  int graph_kernels = 0;
  int loaded = 0;
  int failed = 0;
  int gevd_mode = kDefaultGevdMode;  // FCA_GEVD_FP32 or FCA_GEVD_REFINED
  int max_sweeps = kDefaultSweeps;
  int last_form = -1, last_iters = 0;  // of the last fca_batch_run
};

namespace {

void release(fca_batch* b) {
  for (BatchClass& c : b->cls) {
    void* ptrs[] = {c.bins, c.sample, c.mix_b0, c.mix_nb, c.mix_id, c.vfloor, c.S0, c.S,
                    c.S_prev, c.P, c.lam, c.ldet, c.P_prev, c.lam_prev, c.ldet_prev, c.sep_PH,
                    c.sep_PinvH, c.sep_lam, c.llf};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
  }
  b->cls.clear();
  void* ptrs[] = {b->y, b->v0f, b->v, b->v_prev, b->status};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
}

bool batch_problem_ok(const fca_batch_problem* p) {
  if (!p || p->count < 1 || !p->M || !p->F || !p->N || !p->y || !p->v0 || !p->S0) return false;
  if (p->location != FCA_MEM_DEVICE && p->location != FCA_MEM_HOST) return false;
  for (int k = 0; k < p->count; ++k) {
    if (p->M[k] < 1 || p->M[k] > 8 || p->F[k] < 1 || p->N[k] < 1) return false;
    if ((int64_t)p->F[k] * p->N[k] * p->M[k] >= ((int64_t)1 << 31)) return false;
  }
  return true;
}

// Drop the cached graph (its launch shapes or buffers no longer hold).
void drop_graph(fca_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->key = GraphKey();
  b->graph_kernels = 0;
}

cudaError_t ensure_llf(BatchClass& c, int iters) {
  if (iters <= c.llf_cap) return cudaSuccess;
  if (c.llf) cudaFree(c.llf);
  c.llf = nullptr;
  c.llf_cap = 0;
  cudaError_t e = balloc(&c.llf, (size_t)iters * c.nbins);
  if (e == cudaSuccess) c.llf_cap = iters;
  return e;
}

FastEmArgs fast_args(fca_batch* b, BatchClass& c, int iters, const BinDesc* bins, int nbins) {
  FastEmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = c.nbins;
  a.N = c.Nmax;
  a.iters = iters;
  a.res_bytes = c.res_bytes;
  a.bins = bins;
  a.nbins = nbins;
  a.y = b->y;
  a.ginv = nullptr;
  a.vfloor = c.vfloor;
  a.v_in = b->v0f;
  a.v = b->v;
  a.v_prev = b->v_prev;
  a.P = c.P;
  a.lam = c.lam;
  a.logdetS2 = c.ldet;
  a.P_prev = c.P_prev;
  a.lam_prev = c.lam_prev;
  a.logdetS2_prev = c.ldet_prev;
  a.llf = c.llf;
  a.status = b->status;
  a.max_sweeps = b->max_sweeps;
  a.gevd_mode = b->gevd_mode;
  return a;
}

ParamArgs param_args(fca_batch* b, BatchClass& c) {
  ParamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = c.nbins;
  a.status = b->status;
  a.max_sweeps = b->max_sweeps;
  a.gevd_mode = b->gevd_mode;
  return a;
}

// Threads per CTA the fused FastFCA kernel of a batch supports in the current mode (the
// refined mode needs three warps).
bool batch_threads_ok(const fca_batch* b, int threads) {
  if (threads == 128 || threads == 256) return true;
  return threads == 64 && b->gevd_mode == FCA_GEVD_FP32;
}

// Enqueue the whole job on `st` (classes forked onto their own streams and joined back).
// Returns the number of kernels enqueued in *kernels.
cudaError_t enqueue_job(fca_batch* b, int form, int iters, double* ll, void* x1, void* x2,
                        float* v_out, cudaStream_t st, int* kernels) {
  int nk = 0;
  cudaError_t e = cudaEventRecord(b->fork, st);
  if (e != cudaSuccess) return e;
  for (BatchClass& c : b->cls) {
    if ((e = cudaStreamWaitEvent(c.stream, b->fork, 0)) != cudaSuccess) return e;
    cudaStream_t cs = c.stream;
    const float* v_sep = iters > 0 ? b->v_prev : b->v0f;
    if (form == FCA_FORM_FAST) {
      ParamArgs pa = param_args(b, c);
      pa.S = c.S0;
      pa.P = c.P;
      pa.lam = c.lam;
      pa.logdetS2 = c.ldet;
      if ((e = launch_gevd_from_S(c.M, pa, cs)) != cudaSuccess) return e;
      ++nk;
      if (iters > 0) {
        FastEmArgs a = fast_args(b, c, iters, c.bins, c.nbins);
        if ((e = launch_fast_em(c.M, 0, a, cs, c.threads)) != cudaSuccess) return e;
        ++nk;
      }
      ParamArgs sp = param_args(b, c);
      sp.P = iters > 0 ? c.P_prev : c.P;
      sp.lam = iters > 0 ? c.lam_prev : c.lam;
      sp.PH = c.sep_PH;
      sp.PinvH = c.sep_PinvH;
      sp.lam32 = c.sep_lam;
      if ((e = launch_sep_prep(c.M, sp, cs)) != cudaSuccess) return e;
      ++nk;
      SepFastArgs s;
      std::memset(&s, 0, sizeof(s));
      s.F = c.nbins;
      s.N = c.Nmax;
      s.bins = c.bins;
      s.y = b->y;
      s.v = v_sep;
      s.PH = c.sep_PH;
      s.PinvH = c.sep_PinvH;
      s.lam = c.sep_lam;
      s.x1 = static_cast<float2*>(x1);
      s.x2 = static_cast<float2*>(x2);
      if ((e = launch_sep_fast(c.M, 0, s, cs)) != cudaSuccess) return e;
      ++nk;
    } else {
      if (iters > 0) {
        ConvEmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.F = c.nbins;
        a.N = c.Nmax;
        a.iters = iters;
        a.res_bytes = resident_bytes(c, kResidentCap);
        a.bins = c.bins;
        a.nbins = c.nbins;
        a.y = b->y;
        a.vfloor = c.vfloor;
        a.v_in = b->v0f;
        a.v = b->v;
        a.v_prev = b->v_prev;
        a.S_in = c.S0;
        a.S = c.S;
        a.S_prev = c.S_prev;
        a.llf = c.llf;
        a.status = b->status;
        if ((e = launch_conv_em(c.M, 0, a, cs)) != cudaSuccess) return e;
        ++nk;
      }
      SepConvArgs s;
      std::memset(&s, 0, sizeof(s));
      s.F = c.nbins;
      s.N = c.Nmax;
      s.bins = c.bins;
      s.y = b->y;
      s.v = v_sep;
      s.S = iters > 0 ? c.S_prev : c.S0;
      s.x1 = static_cast<float2*>(x1);
      s.x2 = static_cast<float2*>(x2);
      s.status = b->status;
      if ((e = launch_sep_conv(c.M, 0, s, cs)) != cudaSuccess) return e;
      ++nk;
    }
    if (ll && iters > 0) {
      if ((e = launch_ll_ranges((int)c.mix.size(), iters, c.nbins, c.llf, c.mix_b0, c.mix_nb,
                                c.mix_id, ll, cs)) != cudaSuccess)
        return e;
      ++nk;
    }
    if ((e = cudaEventRecord(c.done, cs)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, c.done, 0)) != cudaSuccess) return e;
  }
  if (v_out) {
    const float* src = iters > 0 ? b->v : b->v0f;
    if ((e = cudaMemcpyAsync(v_out, src, (size_t)b->v_elems * sizeof(float),
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
  }
  *kernels = nk;
  return cudaSuccess;
}

}  // namespace

extern "C" {

fca_status fca_batch_init(const fca_batch_problem* p, void* stream, fca_batch** out) {
  if (!out) return FCA_ERR_ARG;
  *out = nullptr;
  if (!batch_problem_ok(p)) return FCA_ERR_ARG;
  int dev = 0;
  B_CHECK(cudaGetDevice(&dev));
  fca_batch* b = new (std::nothrow) fca_batch;
  if (!b) return FCA_ERR_NOMEM;
  b->count = p->count;
  b->device = dev;
  b->M.assign(p->M, p->M + p->count);
  b->F.assign(p->F, p->F + p->count);
  b->N.assign(p->N, p->N + p->count);
  for (int k = 0; k < b->count; ++k) {
    const long long fnm = (long long)b->F[k] * b->N[k] * b->M[k];
    b->x_off.push_back(b->x_elems);
    b->y_off.push_back(b->y_elems);
    b->v_off.push_back(b->v_elems);
    b->S_off.push_back(b->S_elems);
    b->x_elems += fnm;
    b->y_elems += (fnm + 1) & ~1LL;  // next mixture on a 16-byte boundary
    b->v_elems += 2LL * b->F[k] * b->N[k];
    b->S_elems += 2LL * b->F[k] * b->M[k] * b->M[k];
  }
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(cudaMalloc(&b->y, (size_t)b->y_elems * 8 + 16));
  A(balloc(&b->v0f, (size_t)b->v_elems));
  A(balloc(&b->v, (size_t)b->v_elems));
  A(balloc(&b->v_prev, (size_t)b->v_elems));
  A(balloc(&b->status, 1));
  A(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  A(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  // Classes by channel count, the most work first.
  for (int m = 1; m <= 8 && e == cudaSuccess; ++m) {
    BatchClass c;
    c.M = m;
    for (int k = 0; k < b->count; ++k) {
      if (b->M[k] != m) continue;
      c.mix.push_back(k);
      c.b0.push_back(c.nbins);
      for (int f = 0; f < b->F[k]; ++f) {
        BinDesc d;
        d.y_off = b->y_off[k] + (long long)f * b->N[k] * m;
        d.x_off = b->x_off[k] + (long long)f * b->N[k] * m;
        d.v1_off = b->v_off[k] + (long long)f * b->N[k];
        d.v2_off = b->v_off[k] + (long long)b->F[k] * b->N[k] + (long long)f * b->N[k];
        d.N = b->N[k];
        d.b = c.nbins + f;
        c.host_bins.push_back(d);
      }
      c.nbins += b->F[k];
      c.Nmax = std::max(c.Nmax, b->N[k]);
    }
    if (c.nbins == 0) continue;
    std::stable_sort(c.host_bins.begin(), c.host_bins.end(),
                     [](const BinDesc& x, const BinDesc& y) { return x.N > y.N; });
    b->cls.push_back(c);
  }
  std::stable_sort(b->cls.begin(), b->cls.end(), [](const BatchClass& x, const BatchClass& y) {
    double wx = 0, wy = 0;
    for (const BinDesc& d : x.host_bins) wx += (double)d.N * x.M * x.M;
    for (const BinDesc& d : y.host_bins) wy += (double)d.N * y.M * y.M;
    return wx > wy;
  });
  for (BatchClass& c : b->cls) {
    if (e != cudaSuccess) break;
    const size_t nb = c.nbins, mm = (size_t)c.M * c.M, nm = c.mix.size();
    A(balloc(&c.bins, nb));
    A(balloc(&c.mix_b0, nm));
    A(balloc(&c.mix_nb, nm));
    A(balloc(&c.mix_id, nm));
    A(balloc(&c.vfloor, nb));
    A(balloc(&c.S0, 2 * nb * mm));
    A(balloc(&c.S, 2 * nb * mm));
    A(balloc(&c.S_prev, 2 * nb * mm));
    A(balloc(&c.P, nb * mm));
    A(balloc(&c.lam, nb * c.M));
    A(balloc(&c.ldet, nb));
    A(balloc(&c.P_prev, nb * mm));
    A(balloc(&c.lam_prev, nb * c.M));
    A(balloc(&c.ldet_prev, nb));
    A(balloc(&c.sep_PH, nb * mm));
    A(balloc(&c.sep_PinvH, nb * mm));
    A(balloc(&c.sep_lam, nb * c.M));
    A(ensure_llf(c, 64));
    A(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    A(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    if (e != cudaSuccess) break;
    std::vector<int> nbv, idv;
    for (size_t i = 0; i < nm; ++i) {
      nbv.push_back(b->F[c.mix[i]]);
      idv.push_back(c.mix[i]);
    }
    // Descriptor tables and ranges are copied synchronously (they are tiny and the host
    // vectors are reused afterwards).
    A(cudaMemcpy(c.bins, c.host_bins.data(), nb * sizeof(BinDesc), cudaMemcpyHostToDevice));
    A(cudaMemcpy(c.mix_b0, c.b0.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(c.mix_nb, nbv.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(c.mix_id, idv.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
    c.threads = 128;
    c.res_bytes = resident_bytes(c, kResidentCap);
  }
  if (e != cudaSuccess) {
    release(b);
    delete b;
    cudaGetLastError();
    return cuda_status(e);
  }
  const fca_status rc = fca_batch_load(b, p, stream);
  if (rc != FCA_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    release(b);
    delete b;
    return rc;
  }
  *out = b;
  return FCA_OK;
}

fca_status fca_batch_load(fca_batch* b, const fca_batch_problem* p, void* stream) {
  if (!b || !batch_problem_ok(p) || p->count != b->count) return FCA_ERR_ARG;
  for (int k = 0; k < b->count; ++k)
    if (p->M[k] != b->M[k] || p->F[k] != b->F[k] || p->N[k] != b->N[k]) return FCA_ERR_ARG;
  DeviceGuard guard(b->device);
  if (p->location == FCA_MEM_DEVICE &&
      (!on_device(p->y, b->device) || !on_device(p->v0, b->device) || !on_device(p->S0, b->device)))
    return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const char* ysrc = static_cast<const char*>(p->y);
  if (b->y_elems == b->x_elems) {
    B_CHECK(cudaMemcpyAsync(b->y, ysrc, (size_t)b->x_elems * 8, cudaMemcpyDefault, st));
  } else {
    for (int k = 0; k < b->count; ++k)
      B_CHECK(cudaMemcpyAsync(static_cast<char*>(b->y) + b->y_off[k] * 8, ysrc + b->x_off[k] * 8,
                              (size_t)b->F[k] * b->N[k] * b->M[k] * 8, cudaMemcpyDefault, st));
  }
  const double2* S0 = reinterpret_cast<const double2*>(p->S0);
  for (BatchClass& c : b->cls) {
    const size_t mm = (size_t)c.M * c.M;
    for (size_t i = 0; i < c.mix.size(); ++i) {
      const int k = c.mix[i];
      for (int j = 0; j < 2; ++j)
        B_CHECK(cudaMemcpyAsync(c.S0 + ((size_t)j * c.nbins + c.b0[i]) * mm,
                                S0 + b->S_off[k] + (size_t)j * b->F[k] * mm,
                                (size_t)b->F[k] * mm * sizeof(double2), cudaMemcpyDefault, st));
    }
  }
  const double* v0 = p->v0;
  double* stage = nullptr;
  if (p->location == FCA_MEM_HOST) {
    B_CHECK(cudaMallocAsync((void**)&stage, (size_t)b->v_elems * sizeof(double) + 16, st));
    B_CHECK(cudaMemcpyAsync(stage, p->v0, (size_t)b->v_elems * sizeof(double), cudaMemcpyDefault, st));
    v0 = stage;
  }
  B_CHECK(cudaMemsetAsync(b->status, 0, sizeof(int), st));
  for (BatchClass& c : b->cls) {
    B_CHECK(launch_prepare(c.M, 0, c.nbins, 0, b->y, nullptr, v0, b->v0f, c.vfloor, b->status,
                           st, c.bins));
    note_launches(1);
  }
  if (stage) B_CHECK(cudaFreeAsync(stage, st));
  b->loaded = 1;
  b->failed = 0;
  return FCA_OK;
}

fca_status fca_batch_run(fca_batch* b, int32_t form, int32_t iters, double* loglik_dev,
                         void* x1_dev, void* x2_dev, float* v_dev, int32_t use_graph,
                         void* stream) {
  if (!b || iters < 0 || iters > 65535 || !x1_dev || !x2_dev) return FCA_ERR_ARG;
  if (form != FCA_FORM_FAST && form != FCA_FORM_CONVENTIONAL) return FCA_ERR_ARG;
  if (b->failed || !b->loaded) return FCA_ERR_STATE;
  DeviceGuard guard(b->device);
  if (!on_device(x1_dev, b->device) || !on_device(x2_dev, b->device)) return FCA_ERR_ARG;
  if (loglik_dev && !on_device(loglik_dev, b->device)) return FCA_ERR_ARG;
  if (v_dev && !on_device(v_dev, b->device)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  for (BatchClass& c : b->cls) B_CHECK(ensure_llf(c, iters > 0 ? iters : 1));
  b->last_form = form;
  b->last_iters = iters;
  if (!use_graph) {
    int nk = 0;
    B_CHECK(enqueue_job(b, form, iters, loglik_dev, x1_dev, x2_dev, v_dev, st, &nk));
    note_launches(nk);
    return FCA_OK;
  }
  GraphKey key;
  key.form = form;
  key.iters = iters;
  key.ll = loglik_dev;
  key.x1 = x1_dev;
  key.x2 = x2_dev;
  key.v = v_dev;
  if (!b->exec || !(b->key == key)) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    B_CHECK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int nk = 0;
    const cudaError_t ej = enqueue_job(b, form, iters, loglik_dev, x1_dev, x2_dev, v_dev, b->cap, &nk);
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
    if (ej != cudaSuccess || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cuda_status(ej != cudaSuccess ? ej : ec);
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      b->exec = nullptr;
      return cuda_status(ei);
    }
    b->key = key;
    b->graph_kernels = nk;
  }
  B_CHECK(cudaGraphLaunch(b->exec, st));
  note_launches(b->graph_kernels);
  return FCA_OK;
}

fca_status fca_batch_tune(fca_batch* b, int32_t iters, void* stream) {
  if (!b || iters < 0) return FCA_ERR_ARG;
  if (b->failed || !b->loaded) return FCA_ERR_STATE;
  DeviceGuard guard(b->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int it = std::max(1, std::min((int)iters, 4));
  cudaEvent_t t0, t1;
  B_CHECK(cudaEventCreate(&t0));
  B_CHECK(cudaEventCreate(&t1));
  fca_status rc = FCA_OK;
  for (BatchClass& c : b->cls) {
    if (ensure_llf(c, it) != cudaSuccess) {
      rc = FCA_ERR_NOMEM;
      break;
    }
    // Sample: every k-th bin of the longest-first order (at most 8192 bins), so the sample
    // spans the class's range of lengths.
    const int k = std::max(1, (c.nbins + 8191) / 8192);
    std::vector<BinDesc> smp;
    for (int i = 0; i < c.nbins; i += k) smp.push_back(c.host_bins[i]);
    if (c.sample) cudaFree(c.sample);
    c.sample = nullptr;
    if (balloc(&c.sample, smp.size()) != cudaSuccess ||
        cudaMemcpy(c.sample, smp.data(), smp.size() * sizeof(BinDesc), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      rc = FCA_ERR_CUDA;
      break;
    }
    c.nsample = (int)smp.size();
    ParamArgs pa = param_args(b, c);
    pa.S = c.S0;
    pa.P = c.P;
    pa.lam = c.lam;
    pa.logdetS2 = c.ldet;
    if (launch_gevd_from_S(c.M, pa, st) != cudaSuccess) {
      rc = FCA_ERR_CUDA;
      break;
    }
    note_launches(1);
    // Candidates: threads per CTA x the largest on-chip need admitted under each cap.
    struct Cand {
      int nt, rb;
      float best;
    };
    std::vector<Cand> cands;
    const int threads[] = {64, 128, 256};
    const size_t caps[] = {0, 48 * 1024, 100 * 1024, 200 * 1024};
    for (int nt : threads) {
      if (!batch_threads_ok(b, nt)) continue;
      std::vector<int> tried;
      for (size_t cap : caps) {
        const int rb = resident_bytes(c, cap);
        if (std::find(tried.begin(), tried.end(), rb) != tried.end()) continue;
        tried.push_back(rb);
        cands.push_back({nt, rb, 3.0e38f});
      }
    }
    // One warm-up round, then four timed rounds over all candidates in turn (a drift of the
    // clocks during tuning then affects every candidate alike); each keeps its best time.
    for (int rep = 0; rep < 5; ++rep) {
      for (Cand& cd : cands) {
        if (cd.best < 0.f) continue;  // failed to launch
        FastEmArgs a = fast_args(b, c, it, c.sample, c.nsample);
        a.res_bytes = cd.rb;
        cudaEventRecord(t0, st);
        const cudaError_t e = launch_fast_em(c.M, 0, a, st, cd.nt);
        cudaEventRecord(t1, st);
        float ms = 0.f;
        if (e != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) {
          cudaGetLastError();
          cd.best = -1.f;
          continue;
        }
        note_launches(1);
        if (rep > 0) cd.best = std::min(cd.best, ms);
      }
    }
    int best_t = c.threads, best_r = c.res_bytes;
    float best_ms = 3.0e38f;
    for (const Cand& cd : cands) {
      if (cd.best >= 0.f && cd.best < best_ms) {
        best_ms = cd.best;
        best_t = cd.nt;
        best_r = cd.rb;
      }
    }
    c.threads = best_t;
    c.res_bytes = best_r;
    c.tuned = 1;
  }
  // The groups of a job run at the same time and share the SMs, so the per-group choices are
  // checked together: the tuned shapes, the default shapes (128 threads, bins of up to 100 KB
  // on chip) and the tuned thread counts with every bin streaming each run all groups'
  // EM kernels at once (fork/join over the group streams); the fastest set is kept.
  if (rc == FCA_OK && b->cls.size() > 1) {
    struct Shape {
      int nt, rb;
    };
    std::vector<std::vector<Shape>> sets(3);
    for (BatchClass& c : b->cls) {
      sets[0].push_back({c.threads, c.res_bytes});
      sets[1].push_back({128, resident_bytes(c, kResidentCap)});
      sets[2].push_back({c.threads, 0});
    }
    float best = 3.0e38f;
    int best_set = 0;
    for (int rep = 0; rep < 3 && rc == FCA_OK; ++rep) {
      for (int si = 0; si < 3; ++si) {
        cudaEventRecord(t0, st);
        cudaEventRecord(b->fork, st);
        bool ok = true;
        for (size_t ci = 0; ci < b->cls.size(); ++ci) {
          BatchClass& c = b->cls[ci];
          cudaStreamWaitEvent(c.stream, b->fork, 0);
          FastEmArgs a = fast_args(b, c, it, c.bins, c.nbins);
          a.res_bytes = sets[si][ci].rb;
          if (launch_fast_em(c.M, 0, a, c.stream, sets[si][ci].nt) != cudaSuccess) ok = false;
          else note_launches(1);
          cudaEventRecord(c.done, c.stream);
          cudaStreamWaitEvent(st, c.done, 0);
        }
        cudaEventRecord(t1, st);
        float ms = 0.f;
        if (!ok || cudaEventSynchronize(t1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        if (rep > 0 && ms < best) {  // the first round is a warm-up
          best = ms;
          best_set = si;
        }
      }
    }
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
      b->cls[ci].threads = sets[best_set][ci].nt;
      b->cls[ci].res_bytes = sets[best_set][ci].rb;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  drop_graph(b);
  // The timing runs continue the EM of the sample from one candidate to the next, far past
  // the iterations asked for; what they record in the status word is not a result of the
  // batch, so it is cleared (fca_batch_run starts again from the loaded inputs).
  if (rc == FCA_OK) {
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaMemsetAsync(b->status, 0, sizeof(int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = FCA_ERR_CUDA;
  }
  return rc;
}

fca_status fca_batch_shape(const fca_batch* b, int32_t M, int32_t* bins, int32_t* threads,
                           int32_t* res_bytes) {
  if (!b) return FCA_ERR_ARG;
  for (const BatchClass& c : b->cls) {
    if (c.M != M) continue;
    if (bins) *bins = c.nbins;
    if (threads) *threads = c.threads;
    if (res_bytes) *res_bytes = c.res_bytes;
    return FCA_OK;
  }
  return FCA_ERR_ARG;
}

fca_status fca_batch_set_shape(fca_batch* b, int32_t M, int32_t threads, int32_t res_bytes) {
  if (!b || !batch_threads_ok(b, threads) || res_bytes < 0 || res_bytes > 200 * 1024)
    return FCA_ERR_ARG;
  for (BatchClass& c : b->cls) {
    if (c.M != M) continue;
    c.threads = threads;
    c.res_bytes = res_bytes;
    drop_graph(b);
    return FCA_OK;
  }
  return FCA_ERR_ARG;
}

fca_status fca_batch_get_params(fca_batch* b, int32_t k, double* S_host, double* llf_host,
                                void* stream) {
  if (!b || k < 0 || k >= b->count || (!S_host && !llf_host)) return FCA_ERR_ARG;
  if (b->failed || b->last_form < 0) return FCA_ERR_STATE;
  if (llf_host && b->last_iters <= 0) return FCA_ERR_STATE;
  DeviceGuard guard(b->device);
  cudaStream_t st = (cudaStream_t)stream;
  BatchClass* cp = nullptr;
  int li = -1;
  for (BatchClass& c : b->cls) {
    for (size_t i = 0; i < c.mix.size(); ++i)
      if (c.mix[i] == k) {
        cp = &c;
        li = (int)i;
      }
  }
  if (!cp) return FCA_ERR_ARG;
  BatchClass& c = *cp;
  const size_t Fk = (size_t)b->F[k], MM = (size_t)c.M * c.M, b0 = (size_t)c.b0[li];
  if (S_host) {
    // conventional: the last M-step's S (the initial S0 after a run of zero iterations)
    const double2* src = b->last_iters > 0 ? c.S : c.S0;
    double2* tmp = nullptr;
    if (b->last_form == FCA_FORM_FAST) {  // S_j = P^-H T_j P^-1 of the class's bins
      B_CHECK(balloc(&tmp, 2 * (size_t)c.nbins * MM));
      ParamArgs pa = param_args(b, c);
      pa.P = c.P;
      pa.lam = c.lam;
      pa.S_out = tmp;
      const cudaError_t e = launch_S_from_P(c.M, pa, st);
      if (e != cudaSuccess) {
        cudaFree(tmp);
        return cuda_status(e);
      }
      note_launches(1);
      src = tmp;
    }
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < 2 && e == cudaSuccess; ++j)
      e = cudaMemcpyAsync(S_host + 2 * (size_t)j * Fk * MM, src + ((size_t)j * c.nbins + b0) * MM,
                          Fk * MM * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    B_CHECK(e);
  }
  if (llf_host) {
    B_CHECK(cudaMemcpy2DAsync(llf_host, Fk * sizeof(double), c.llf + b0, (size_t)c.nbins * sizeof(double),
                              Fk * sizeof(double), (size_t)b->last_iters, cudaMemcpyDeviceToHost, st));
    B_CHECK(cudaStreamSynchronize(st));
  }
  return FCA_OK;
}

fca_status fca_batch_set_eigensolver(fca_batch* b, int32_t precision, int32_t max_sweeps) {
  if (!b || (precision != FCA_GEVD_FP32 && precision != FCA_GEVD_REFINED) || max_sweeps < 0 ||
      max_sweeps > FCA_MAX_SWEEPS_LIMIT)
    return FCA_ERR_ARG;
  if (precision != b->gevd_mode) {
    // Launch shapes tuned for the other mode no longer apply.
    for (BatchClass& c : b->cls) {
      c.threads = 128;
      c.res_bytes = resident_bytes(c, kResidentCap);
      c.tuned = 0;
    }
  }
  b->gevd_mode = precision;
  b->max_sweeps = max_sweeps;
  drop_graph(b);
  return FCA_OK;
}

fca_status fca_batch_sync_status(fca_batch* b, void* stream) {
  if (!b) return FCA_ERR_ARG;
  DeviceGuard guard(b->device);
  B_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
  int code = 0;
  B_CHECK(cudaMemcpy(&code, b->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (code != 0) {
    b->failed = 1;
    return (fca_status)code;
  }
  return FCA_OK;
}

void fca_batch_free(fca_batch* b) {
  if (!b) return;
  {
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    release(b);
  }
  delete b;
}

}  // extern "C"
