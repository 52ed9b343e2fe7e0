// FastFCA without any device allocation: the whole job of fca_em_fast on caller-owned
// inputs and outputs, with the library's scratch in one fixed, file-scope device array.
//
// Who needs it: callers that must not allocate device memory once they are running -- a
// real-time audio loop (cudaMalloc / cudaFree may synchronise the device and take an
// unbounded time), or a host application that hands out device memory only through its own
// pool and forbids allocations by the libraries it loads. The paper has no counterpart: this
// is a deployment variant of the same kernels.
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "fca.h"
#include "fca_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)FCA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits. Host code must
// not pass the symbol itself to a kernel: on the host it is only a stand-in; the device
// address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

// Device address of the scratch array for the current device (set up on the first call on
// that device, with that device current).
cudaError_t scratch_for_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned char* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    p = static_cast<unsigned char*>(addr);
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return cudaSuccess;
}

struct Layout {  // byte offsets into the scratch array, each 256-byte aligned
  size_t status, vfloor, P, lam, ldet, P_prev, lam_prev, ldet_prev, llf, v_prev, sep_PH, sep_PinvH,
      sep_lam, total;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int M, int F, int N, int iters) {
  Layout L;
  const size_t f = (size_t)F, mm = (size_t)M * M;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += up256(bytes);
    return at;
  };
  L.status = take(sizeof(int));
  L.vfloor = take(f * sizeof(float));
  L.P = take(f * mm * sizeof(double2));
  L.lam = take(f * M * sizeof(double));
  L.ldet = take(f * sizeof(double));
  L.P_prev = take(f * mm * sizeof(double2));
  L.lam_prev = take(f * M * sizeof(double));
  L.ldet_prev = take(f * sizeof(double));
  L.llf = take((size_t)(iters > 0 ? iters : 1) * f * sizeof(double));
  L.v_prev = take(2 * f * N * sizeof(float));
  L.sep_PH = take(f * mm * sizeof(float2));
  L.sep_PinvH = take(f * mm * sizeof(float2));
  L.sep_lam = take(f * M * sizeof(float));
  L.total = o;
  return L;
}

bool aligned(const void* ptr, size_t a) { return reinterpret_cast<uintptr_t>(ptr) % a == 0; }

bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" fca_status fca_em_fast_noalloc(int32_t M, int32_t F, int32_t N, const void* y_dev,
                                          const double* v0_dev, const double* S0_dev,
                                          int32_t iters, float* v_dev, void* x1_dev,
                                          void* x2_dev, double* loglik_dev, void* stream) {
  if (M < 1 || M > 8 || F < 1 || N < 1 || iters < 0) return FCA_ERR_ARG;
  if ((int64_t)F * N * M >= ((int64_t)1 << 31)) return FCA_ERR_ARG;
  if (!y_dev || !v0_dev || !S0_dev || !v_dev || !x1_dev || !x2_dev) return FCA_ERR_ARG;
  const Layout L = layout(M, F, N, iters);
  if (L.total > kScratchBytes) return FCA_ERR_SCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FCA_ERR_CUDA;
  const void* ptrs[] = {y_dev, v0_dev, S0_dev, v_dev, x1_dev, x2_dev};
  for (const void* q : ptrs)
    if (!on_device(q, dev)) return FCA_ERR_ARG;
  if (loglik_dev && !on_device(loglik_dev, dev)) return FCA_ERR_ARG;
  // The kernels read the caller's buffers in place with vector loads (no staging copy as in
  // fca_init): y and S0 by 16 bytes, v0 and the outputs by their element size.
  if (!aligned(y_dev, 16) || !aligned(S0_dev, 16) || !aligned(v0_dev, 8) || !aligned(v_dev, 4) ||
      !aligned(x1_dev, 8) || !aligned(x2_dev, 8) || (loglik_dev && !aligned(loglik_dev, 8)))
    return FCA_ERR_ARG;
  unsigned char* base = nullptr;
  if (scratch_for_device(dev, &base) != cudaSuccess) return FCA_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  int* status = reinterpret_cast<int*>(base + L.status);
  float* vfloor = reinterpret_cast<float*>(base + L.vfloor);
  double2* P = reinterpret_cast<double2*>(base + L.P);
  double* lam = reinterpret_cast<double*>(base + L.lam);
  double* ldet = reinterpret_cast<double*>(base + L.ldet);
  double2* P_prev = reinterpret_cast<double2*>(base + L.P_prev);
  double* lam_prev = reinterpret_cast<double*>(base + L.lam_prev);
  double* ldet_prev = reinterpret_cast<double*>(base + L.ldet_prev);
  double* llf = reinterpret_cast<double*>(base + L.llf);
  float* v_prev = reinterpret_cast<float*>(base + L.v_prev);

#define NA_CHECK(expr)                                                       \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? FCA_ERR_NOMEM : FCA_ERR_CUDA; \
  } while (0)

  // The array keeps the previous call's contents: the status word must start at zero; every
  // other region is written before it is read.
  NA_CHECK(cudaMemsetAsync(status, 0, sizeof(int), st));
  // One pass: the floor and initial v, and the generalised eigenproblem of S0 (Eq. (GEVD)).
  fca::PrepareExtra ex = {};
  ex.max_sweeps = fca::kDefaultSweeps;
  ex.gevd_mode = fca::kDefaultGevdMode;
  ex.S = reinterpret_cast<const double2*>(S0_dev);
  ex.P = P;
  ex.lam = lam;
  ex.logdetS2 = ldet;
  NA_CHECK(fca::launch_prepare(M, FCA_STORE_C64, F, N, y_dev, nullptr, v0_dev, v_dev, vfloor, status, st,
                               nullptr, &ex));
  fca::note_launches(1);
  if (iters > 0) {
    fca::FastEmArgs a = {};
    a.F = F;
    a.N = N;
    a.iters = iters;
    a.res_bytes = fca::em_resident(M, FCA_STORE_C64, N) ? (int)fca::em_dyn_smem(M, FCA_STORE_C64, N) : 0;
    a.bins = nullptr;
    a.y = y_dev;
    a.ginv = nullptr;
    a.vfloor = vfloor;
    a.v_in = v_dev;
    a.v = v_dev;
    a.v_prev = v_prev;
    a.P = P;
    a.lam = lam;
    a.logdetS2 = ldet;
    a.P_prev = P_prev;
    a.lam_prev = lam_prev;
    a.logdetS2_prev = ldet_prev;
    a.llf = llf;
    a.status = status;
    a.max_sweeps = fca::kDefaultSweeps;
    a.gevd_mode = fca::kDefaultGevdMode;
    NA_CHECK(fca::launch_fast_em(M, FCA_STORE_C64, a, st));
    fca::note_launches(1);
    if (loglik_dev) {
      NA_CHECK(fca::launch_ll_reduce(F, iters, llf, loglik_dev, st));
      fca::note_launches(1);
    }
  }
  // Algorithm 1's output: the E-step of iteration L-1 (the initial parameters when L = 0).
  fca::ParamArgs sp = {};
  sp.F = F;
  sp.status = status;
  sp.P = iters > 0 ? P_prev : P;
  sp.lam = iters > 0 ? lam_prev : lam;
  sp.ginv = nullptr;
  sp.PH = reinterpret_cast<float2*>(base + L.sep_PH);
  sp.PinvH = reinterpret_cast<float2*>(base + L.sep_PinvH);
  sp.lam32 = reinterpret_cast<float*>(base + L.sep_lam);
  NA_CHECK(fca::launch_sep_prep(M, sp, st));
  fca::note_launches(1);
  fca::SepFastArgs s = {};
  s.F = F;
  s.N = N;
  s.y = y_dev;
  s.ginv = nullptr;
  s.v = iters > 0 ? v_prev : v_dev;
  s.PH = sp.PH;
  s.PinvH = sp.PinvH;
  s.lam = sp.lam32;
  s.x1 = static_cast<float2*>(x1_dev);
  s.x2 = static_cast<float2*>(x2_dev);
  NA_CHECK(fca::launch_sep_fast(M, FCA_STORE_C64, s, st));
  fca::note_launches(1);
  // Read the status word on the call's own stream (a plain cudaMemcpy would also wait for
  // every other blocking stream of the device).
  int code = 0;
  NA_CHECK(cudaMemcpyAsync(&code, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CHECK(cudaStreamSynchronize(st));
#undef NA_CHECK
  return (fca_status)code;
}
