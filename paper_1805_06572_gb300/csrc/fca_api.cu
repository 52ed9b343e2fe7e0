// C ABI of the FCA library: state ownership, argument checks, form switching and launches.
// See include/fca.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>

#include "fca.h"
#include "fca_internal.h"

using namespace fca;

namespace {

// kFormS: S holds the parameters; kFormP: (P, Lambda) do; kFormSP: both (S0 and its
// generalised eigenproblem, as left by a load).
enum { kFormS = 0, kFormP = 1, kFormSP = 2 };

std::atomic<uint64_t> g_launches{0};

// Every launch_* helper of the kernel files launches exactly one kernel.
cudaError_t counted(cudaError_t e) {
  if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

struct DeviceGuard {  // make the state's device current for the duration of a call
  int old = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DeviceGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

}  // namespace

struct fca_state {
  int M, F, N, storage, device;
  int N_cap;  // frames the device buffers were sized for (fca_init); N <= N_cap
  size_t FN, MM;
  void* y;
  float* g;
  float* ginv;
  float* vfloor;
  float* v;
  float* v_prev;
  double* v0_stage;
  double2* P;
  double* lam;
  double* logdetS2;
  double2* P_prev;
  double* lam_prev;
  double* logdetS2_prev;
  double2* S;
  double2* S_prev;
  double2* S_tmp;
  double* llf;
  int llf_cap;
  int last_iters;  // iterations of the last EM call (0: none since the last load)
  cudaEvent_t ev_em[2];
  int have_events;
  float2* sep_PH;
  float2* sep_PinvH;
  float* sep_lam;
  int* status;
  int form;
  int prev_form;  // -1: no iteration run since the last load
  int failed;
  int gevd_mode;   // FastFCA eigensolver and Gram merge precision (FCA_GEVD_*)
  int max_sweeps;  // Jacobi sweep cap
  int conv_layout; // FCA_CONV_*
};

namespace {

fca_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FCA_OK;
  if (e == cudaErrorMemoryAllocation) return FCA_ERR_NOMEM;
  return FCA_ERR_CUDA;
}

#define FCA_CHECK_CUDA(expr)                          \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_status(e_);    \
  } while (0)

bool problem_ok(const fca_problem* p) {
  if (!p) return false;
  if (p->M < 1 || p->M > 8 || p->F < 1 || p->N < 1) return false;
  if ((int64_t)p->F * p->N * p->M >= ((int64_t)1 << 31)) return false;
  if (p->storage != FCA_STORE_C64 && p->storage != FCA_STORE_F16_SCALED) return false;
  if (p->location != FCA_MEM_DEVICE && p->location != FCA_MEM_HOST) return false;
  if (!p->y || (!p->v0) != (!p->S0)) return false;
  // FP16 storage without a scale: a complex64 mixture on the device, encoded by the library
  if (p->storage == FCA_STORE_F16_SCALED && !p->y_scale && p->location != FCA_MEM_DEVICE) return false;
  return true;
}

bool device_pointer(const void* ptr, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

bool aligned(const void* ptr, size_t a) { return reinterpret_cast<uintptr_t>(ptr) % a == 0; }

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

void release(fca_state* s) {
  if (s->have_events) {
    cudaEventDestroy(s->ev_em[0]);
    cudaEventDestroy(s->ev_em[1]);
    s->have_events = 0;
  }
  void* ptrs[] = {s->y, s->g, s->ginv, s->vfloor, s->v, s->v_prev, s->v0_stage, s->P, s->lam,
                  s->logdetS2, s->P_prev, s->lam_prev, s->logdetS2_prev, s->S, s->S_prev,
                  s->S_tmp, s->llf, s->sep_PH, s->sep_PinvH, s->sep_lam, s->status};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

fca_status ensure_llf(fca_state* s, int iters) {
  if (iters <= s->llf_cap) return FCA_OK;
  if (s->llf) cudaFree(s->llf);
  s->llf = nullptr;
  s->llf_cap = 0;
  FCA_CHECK_CUDA(dalloc(&s->llf, (size_t)iters * s->F));
  s->llf_cap = iters;
  return FCA_OK;
}

ParamArgs param_args(fca_state* s) {
  ParamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = s->F;
  a.status = s->status;
  a.max_sweeps = s->max_sweeps;
  a.gevd_mode = s->gevd_mode;
  return a;
}

}  // namespace

void fca::note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

extern "C" {

const char* fca_status_string(fca_status st) {
  switch (st) {
    case FCA_OK: return "ok";
    case FCA_ERR_ARG: return "invalid argument";
    case FCA_ERR_CUDA: return "CUDA runtime error";
    case FCA_ERR_NOMEM: return "device allocation failed";
    case FCA_ERR_NOT_PD: return "matrix not positive definite";
    case FCA_ERR_EIG_NOCONV: return "eigensolver did not converge";
    case FCA_ERR_NONFINITE: return "non-finite value";
    case FCA_ERR_TIMEOUT: return "device wait timed out";
    case FCA_ERR_STATE: return "state failed earlier or call does not fit its form";
    case FCA_ERR_SCRATCH: return "problem larger than the no-allocation scratch array";
  }
  return "unknown status";
}

const char* fca_version(void) { return "fca-gb300 1.0 (sm_103a)"; }

fca_status fca_load(fca_state* s, const fca_problem* p, void* stream) {
  if (!s || !problem_ok(p)) return FCA_ERR_ARG;
  if (p->M != s->M || p->F != s->F || p->N > s->N_cap || p->storage != s->storage) return FCA_ERR_ARG;
  DeviceGuard guard(s->device);
  const bool seeded = !p->v0;  // with S0 == NULL (problem_ok)
  const bool encode = p->storage == FCA_STORE_F16_SCALED && !p->y_scale;
  if (p->location == FCA_MEM_DEVICE) {
    if (!device_pointer(p->y, s->device) ||
        (!seeded && (!device_pointer(p->v0, s->device) || !device_pointer(p->S0, s->device))) ||
        (p->storage == FCA_STORE_F16_SCALED && !encode && !device_pointer(p->y_scale, s->device)))
      return FCA_ERR_ARG;
    if (encode && !aligned(p->y, 8)) return FCA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  s->N = p->N;
  s->FN = (size_t)s->F * s->N;
  const size_t ybytes = s->FN * s->M * (s->storage ? 4 : 8);
  // Device inputs: the prepare pass copies y and S0 into the state as it reads them. Host
  // inputs: copied up first, then read in place. A mixture the library encodes to FP16 is
  // written into the state by the encoding pass; seeded initial values are written into the
  // state's S and the v0 staging buffer.
  // (Element-misaligned device inputs take the copy route too.)
  const bool on_dev = p->location == FCA_MEM_DEVICE;
  const bool y_direct = on_dev && !encode && aligned(p->y, s->storage ? 4 : 8);
  const bool S_direct = on_dev && !seeded && aligned(p->S0, 16);
  PrepareExtra ex;
  std::memset(&ex, 0, sizeof(ex));
  ex.max_sweeps = s->max_sweeps;
  ex.gevd_mode = s->gevd_mode;
  ex.P = s->P;
  ex.lam = s->lam;
  ex.logdetS2 = s->logdetS2;
  if (encode) {
    FCA_CHECK_CUDA(counted(launch_encode_f16(s->F, s->N * s->M, p->y, s->y, s->g, st)));
  } else if (y_direct) {
    ex.y_copy = s->y;
  } else {
    FCA_CHECK_CUDA(cudaMemcpyAsync(s->y, p->y, ybytes, cudaMemcpyDefault, st));
  }
  if (s->storage == FCA_STORE_F16_SCALED) {
    if (!encode) FCA_CHECK_CUDA(cudaMemcpyAsync(s->g, p->y_scale, s->F * sizeof(float), cudaMemcpyDefault, st));
    FCA_CHECK_CUDA(counted(launch_invert_scale(s->F, s->g, s->ginv, st)));
  }
  if (seeded) {
    if (!s->v0_stage) FCA_CHECK_CUDA(dalloc(&s->v0_stage, 2 * (size_t)s->F * s->N_cap));
    FCA_CHECK_CUDA(counted(launch_seeded_init(s->M, s->storage, s->F, s->N, y_direct ? p->y : s->y, s->g,
                                              (unsigned long long)p->seed, s->S, s->v0_stage, st)));
    ex.S = s->S;
  } else if (S_direct) {
    ex.S = static_cast<const double2*>(static_cast<const void*>(p->S0));
    ex.S_copy = s->S;
  } else {
    FCA_CHECK_CUDA(cudaMemcpyAsync(s->S, p->S0, 2 * s->F * s->MM * sizeof(double2), cudaMemcpyDefault, st));
    ex.S = s->S;
  }
  const double* v0 = seeded ? s->v0_stage : p->v0;
  if (!seeded && (!on_dev || !aligned(p->v0, 8))) {
    if (!s->v0_stage) FCA_CHECK_CUDA(dalloc(&s->v0_stage, 2 * (size_t)s->F * s->N_cap));
    FCA_CHECK_CUDA(cudaMemcpyAsync(s->v0_stage, p->v0, 2 * s->FN * sizeof(double), cudaMemcpyDefault, st));
    v0 = s->v0_stage;
  }
  FCA_CHECK_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  FCA_CHECK_CUDA(counted(launch_prepare(s->M, s->storage, s->F, s->N, y_direct ? p->y : s->y, s->ginv, v0,
                                        s->v, s->vfloor, s->status, st, nullptr, &ex)));
  s->form = kFormSP;
  s->prev_form = -1;
  s->failed = 0;
  s->last_iters = 0;
  return FCA_OK;
}

fca_status fca_init(const fca_problem* p, void* stream, fca_state** out) {
  if (!out) return FCA_ERR_ARG;
  *out = nullptr;
  if (!problem_ok(p)) return FCA_ERR_ARG;
  int dev = 0;
  FCA_CHECK_CUDA(cudaGetDevice(&dev));
  fca_state* s = new (std::nothrow) fca_state;
  if (!s) return FCA_ERR_NOMEM;
  std::memset(s, 0, sizeof(*s));
  s->M = p->M;
  s->F = p->F;
  s->N = p->N;
  s->N_cap = p->N;
  s->storage = p->storage;
  s->device = dev;
  s->gevd_mode = kDefaultGevdMode;
  s->max_sweeps = kDefaultSweeps;
  s->FN = (size_t)p->F * p->N;
  s->MM = (size_t)p->M * p->M;
  const size_t F = s->F, FN = s->FN, MM = s->MM;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(cudaMalloc(&s->y, FN * s->M * (s->storage ? 4 : 8) + 16));
  A(dalloc(&s->g, F));
  A(dalloc(&s->ginv, F));
  A(dalloc(&s->vfloor, F));
  A(dalloc(&s->v, 2 * FN));
  A(dalloc(&s->v_prev, 2 * FN));
  A(dalloc(&s->P, F * MM));
  A(dalloc(&s->lam, F * s->M));
  A(dalloc(&s->logdetS2, F));
  A(dalloc(&s->P_prev, F * MM));
  A(dalloc(&s->lam_prev, F * s->M));
  A(dalloc(&s->logdetS2_prev, F));
  A(dalloc(&s->S, 2 * F * MM));
  A(dalloc(&s->S_prev, 2 * F * MM));
  A(dalloc(&s->S_tmp, 2 * F * MM));
  A(dalloc(&s->sep_PH, F * MM));
  A(dalloc(&s->sep_PinvH, F * MM));
  A(dalloc(&s->sep_lam, F * s->M));
  A(dalloc(&s->status, 1));
  A(cudaEventCreate(&s->ev_em[0]));
  A(cudaEventCreate(&s->ev_em[1]));
  if (e == cudaSuccess) s->have_events = 1;
  if (e == cudaSuccess) {
    s->llf_cap = 0;
    if (ensure_llf(s, 64) != FCA_OK) e = cudaErrorMemoryAllocation;
  }
  if (e != cudaSuccess) {
    release(s);
    delete s;
    cudaGetLastError();
    return cuda_status(e);
  }
  if (p->storage == FCA_STORE_C64) {
    cudaMemsetAsync(s->ginv, 0, F * sizeof(float), (cudaStream_t)stream);
  }
  fca_status rc = fca_load(s, p, stream);
  if (rc != FCA_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    release(s);
    delete s;
    return rc;
  }
  *out = s;
  return FCA_OK;
}

fca_status fca_em_fast(fca_state* s, int32_t iters, double* loglik_dev, void* stream) {
  if (!s || iters < 0) return FCA_ERR_ARG;
  if (s->failed) return FCA_ERR_STATE;
  if (iters == 0) return FCA_OK;
  DeviceGuard guard(s->device);
  if (loglik_dev && !device_pointer(loglik_dev, s->device)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fca_status rc = ensure_llf(s, iters);
  if (rc != FCA_OK) return rc;
  if (s->form == kFormS) {
    ParamArgs pa = param_args(s);
    pa.S = s->S;
    pa.P = s->P;
    pa.lam = s->lam;
    pa.logdetS2 = s->logdetS2;
    FCA_CHECK_CUDA(counted(launch_gevd_from_S(s->M, pa, st)));
  }
  s->form = kFormP;
  FastEmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = s->F;
  a.N = s->N;
  a.iters = iters;
  a.res_bytes = em_resident(s->M, s->storage, s->N) ? (int)em_dyn_smem(s->M, s->storage, s->N) : 0;
  a.bins = nullptr;
  a.y = s->y;
  a.ginv = s->ginv;
  a.vfloor = s->vfloor;
  a.v_in = s->v;
  a.v = s->v;
  a.v_prev = s->v_prev;
  a.P = s->P;
  a.lam = s->lam;
  a.logdetS2 = s->logdetS2;
  a.P_prev = s->P_prev;
  a.lam_prev = s->lam_prev;
  a.logdetS2_prev = s->logdetS2_prev;
  a.llf = s->llf;
  a.status = s->status;
  a.max_sweeps = s->max_sweeps;
  a.gevd_mode = s->gevd_mode;
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[0], st));
  FCA_CHECK_CUDA(counted(launch_fast_em(s->M, s->storage, a, st)));
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[1], st));
  s->prev_form = kFormP;
  s->last_iters = iters;
  if (loglik_dev) FCA_CHECK_CUDA(counted(launch_ll_reduce(s->F, iters, s->llf, loglik_dev, st)));
  return FCA_OK;
}

fca_status fca_em_fast_recover(fca_state* s, int32_t iters, double* loglik_dev, void* stream) {
  if (!s || iters < 0) return FCA_ERR_ARG;
  if (s->failed) return FCA_ERR_STATE;
  if (iters == 0) return FCA_OK;
  DeviceGuard guard(s->device);
  if (loglik_dev && !device_pointer(loglik_dev, s->device)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fca_status rc = ensure_llf(s, iters);
  if (rc != FCA_OK) return rc;
  ParamArgs pa = param_args(s);
  pa.S = s->S;
  pa.P = s->P;
  pa.lam = s->lam;
  pa.logdetS2 = s->logdetS2;
  pa.S_out = s->S;
  if (s->form == kFormS) FCA_CHECK_CUDA(counted(launch_gevd_from_S(s->M, pa, st)));
  s->form = kFormP;
  FastEmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = s->F;
  a.N = s->N;
  a.iters = 1;
  a.res_bytes = em_resident(s->M, s->storage, s->N) ? (int)em_dyn_smem(s->M, s->storage, s->N) : 0;
  a.y = s->y;
  a.ginv = s->ginv;
  a.vfloor = s->vfloor;
  a.v_in = s->v;
  a.v = s->v;
  a.v_prev = s->v_prev;
  a.P = s->P;
  a.lam = s->lam;
  a.logdetS2 = s->logdetS2;
  a.P_prev = s->P_prev;
  a.lam_prev = s->lam_prev;
  a.logdetS2_prev = s->logdetS2_prev;
  a.status = s->status;
  a.max_sweeps = s->max_sweeps;
  a.gevd_mode = s->gevd_mode;
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[0], st));
  for (int l = 0; l < iters; ++l) {
    // One iteration (E-step, M-step in the transformed basis) with the parameters of
    // iteration l; then S_j = P^-H T_j P^-1 (Eqs. (Sdiag), (recoverS)) and (P, Lambda) from
    // the generalised eigenproblem of (S1, S2) afresh (Eq. (GEVD)).
    a.llf = s->llf + (size_t)l * s->F;
    FCA_CHECK_CUDA(counted(launch_fast_em(s->M, s->storage, a, st)));
    FCA_CHECK_CUDA(counted(launch_S_from_P(s->M, pa, st)));
    FCA_CHECK_CUDA(counted(launch_gevd_from_S(s->M, pa, st)));
  }
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[1], st));
  s->prev_form = kFormP;
  s->last_iters = iters;
  if (loglik_dev) FCA_CHECK_CUDA(counted(launch_ll_reduce(s->F, iters, s->llf, loglik_dev, st)));
  return FCA_OK;
}

fca_status fca_em_conventional(fca_state* s, int32_t iters, double* loglik_dev, void* stream) {
  if (!s || iters < 0) return FCA_ERR_ARG;
  if (s->failed) return FCA_ERR_STATE;
  if (iters == 0) return FCA_OK;
  DeviceGuard guard(s->device);
  if (loglik_dev && !device_pointer(loglik_dev, s->device)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fca_status rc = ensure_llf(s, iters);
  if (rc != FCA_OK) return rc;
  if (s->form == kFormP) {
    ParamArgs pa = param_args(s);
    pa.P = s->P;
    pa.lam = s->lam;
    pa.S_out = s->S;
    FCA_CHECK_CUDA(counted(launch_S_from_P(s->M, pa, st)));
  }
  s->form = kFormS;
  ConvEmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.F = s->F;
  a.N = s->N;
  a.iters = iters;
  a.res_bytes = em_resident(s->M, s->storage, s->N) ? (int)em_dyn_smem(s->M, s->storage, s->N) : 0;
  a.bins = nullptr;
  a.y = s->y;
  a.ginv = s->ginv;
  a.vfloor = s->vfloor;
  a.v_in = s->v;
  a.v = s->v;
  a.v_prev = s->v_prev;
  a.S_in = s->S;
  a.S = s->S;
  a.S_prev = s->S_prev;
  a.llf = s->llf;
  a.status = s->status;
  a.layout = s->conv_layout;
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[0], st));
  FCA_CHECK_CUDA(counted(launch_conv_em(s->M, s->storage, a, st)));
  FCA_CHECK_CUDA(cudaEventRecord(s->ev_em[1], st));
  s->prev_form = kFormS;
  s->last_iters = iters;
  if (loglik_dev) FCA_CHECK_CUDA(counted(launch_ll_reduce(s->F, iters, s->llf, loglik_dev, st)));
  return FCA_OK;
}

fca_status fca_separate(fca_state* s, void* x1_dev, void* x2_dev, int32_t mode, void* stream) {
  if (!s || !x1_dev || !x2_dev || (mode != FCA_SEP_ALG1 && mode != FCA_SEP_FINAL_PARAMS))
    return FCA_ERR_ARG;
  if (s->failed) return FCA_ERR_STATE;
  DeviceGuard guard(s->device);
  if (!device_pointer(x1_dev, s->device) || !device_pointer(x2_dev, s->device)) return FCA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const bool use_prev = (mode == FCA_SEP_ALG1 && s->prev_form >= 0);
  const int form = use_prev ? s->prev_form : s->form;
  const float* v = use_prev ? s->v_prev : s->v;
  if (form == kFormP) {
    ParamArgs pa = param_args(s);
    pa.P = use_prev ? s->P_prev : s->P;
    pa.lam = use_prev ? s->lam_prev : s->lam;
    pa.ginv = s->storage ? s->ginv : nullptr;
    pa.PH = s->sep_PH;
    pa.PinvH = s->sep_PinvH;
    pa.lam32 = s->sep_lam;
    FCA_CHECK_CUDA(counted(launch_sep_prep(s->M, pa, st)));
    SepFastArgs a;
    std::memset(&a, 0, sizeof(a));
    a.F = s->F;
    a.N = s->N;
    a.y = s->y;
    a.ginv = s->ginv;
    a.v = v;
    a.PH = s->sep_PH;
    a.PinvH = s->sep_PinvH;
    a.lam = s->sep_lam;
    a.x1 = (float2*)x1_dev;
    a.x2 = (float2*)x2_dev;
    FCA_CHECK_CUDA(counted(launch_sep_fast(s->M, s->storage, a, st)));
  } else {
    SepConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.F = s->F;
    a.N = s->N;
    a.y = s->y;
    a.ginv = s->ginv;
    a.v = v;
    a.S = use_prev ? s->S_prev : s->S;
    a.x1 = (float2*)x1_dev;
    a.x2 = (float2*)x2_dev;
    a.status = s->status;
    FCA_CHECK_CUDA(counted(launch_sep_conv(s->M, s->storage, a, st)));
  }
  return FCA_OK;
}

fca_status fca_get_params(fca_state* s, float* v_dev, double* S_host, void* stream) {
  if (!s) return FCA_ERR_ARG;
  if (s->failed) return FCA_ERR_STATE;
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (v_dev) {
    if (!device_pointer(v_dev, s->device)) return FCA_ERR_ARG;
    FCA_CHECK_CUDA(cudaMemcpyAsync(v_dev, s->v, 2 * s->FN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  if (S_host) {
    const double2* src = s->S;
    if (s->form == kFormP) {
      ParamArgs pa = param_args(s);
      pa.P = s->P;
      pa.lam = s->lam;
      pa.S_out = s->S_tmp;
      FCA_CHECK_CUDA(counted(launch_S_from_P(s->M, pa, st)));
      src = s->S_tmp;
    }
    FCA_CHECK_CUDA(cudaMemcpyAsync(S_host, src, 2 * s->F * s->MM * sizeof(double2), cudaMemcpyDefault, st));
    FCA_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  return FCA_OK;
}

fca_status fca_loglik_bins(fca_state* s, double* out, int32_t* iters_out, void* stream) {
  if (!s || (!out && !iters_out)) return FCA_ERR_ARG;
  if (iters_out) *iters_out = s->last_iters;
  if (s->last_iters <= 0) return FCA_ERR_STATE;
  if (!out) return FCA_OK;
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  FCA_CHECK_CUDA(cudaMemcpyAsync(out, s->llf, (size_t)s->last_iters * s->F * sizeof(double),
                                 cudaMemcpyDefault, st));
  if (!device_pointer(out, s->device)) FCA_CHECK_CUDA(cudaStreamSynchronize(st));
  return FCA_OK;
}

fca_status fca_last_em_kernel_ms(fca_state* s, float* ms) {
  if (!s || !ms) return FCA_ERR_ARG;
  if (s->last_iters <= 0) return FCA_ERR_STATE;
  DeviceGuard guard(s->device);
  FCA_CHECK_CUDA(cudaEventSynchronize(s->ev_em[1]));
  FCA_CHECK_CUDA(cudaEventElapsedTime(ms, s->ev_em[0], s->ev_em[1]));
  return FCA_OK;
}

uint64_t fca_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

fca_status fca_sync_status(fca_state* s, void* stream) {
  if (!s) return FCA_ERR_ARG;
  DeviceGuard guard(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  FCA_CHECK_CUDA(cudaStreamSynchronize(st));
  int code = 0;
  FCA_CHECK_CUDA(cudaMemcpy(&code, s->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (code != 0) {
    s->failed = 1;
    return (fca_status)code;
  }
  return FCA_OK;
}

fca_status fca_set_eigensolver(fca_state* s, int32_t precision, int32_t max_sweeps) {
  if (!s || (precision != FCA_GEVD_FP32 && precision != FCA_GEVD_FP64 && precision != FCA_GEVD_REFINED) ||
      max_sweeps < 0 || max_sweeps > FCA_MAX_SWEEPS_LIMIT)
    return FCA_ERR_ARG;
  s->gevd_mode = precision;
  s->max_sweeps = max_sweeps;
  // A state just loaded holds S0 and the eigenproblem of S0 solved with the old settings: the
  // next fca_em_fast solves it again with these.
  if (s->form == kFormSP) s->form = kFormS;
  return FCA_OK;
}

fca_status fca_set_conv_layout(fca_state* s, int32_t layout) {
  if (!s || (layout != FCA_CONV_AUTO && layout != FCA_CONV_THREAD && layout != FCA_CONV_GROUP))
    return FCA_ERR_ARG;
  s->conv_layout = layout;
  return FCA_OK;
}

void fca_free(fca_state* s) {
  if (!s) return;
  {
    DeviceGuard guard(s->device);
    cudaDeviceSynchronize();
    release(s);
  }
  delete s;
}

}  // extern "C"
