// Allocation-free variant of the projected Tikhonov solve (lslu_projected_noalloc).
//
// Some callers cannot call cudaMalloc: code running under a framework whose
// memory pool must own every device allocation, or a time-critical loop where
// an allocation (with its implicit synchronisation) is not acceptable.  This
// entry point runs the same projected-solve kernel as lslu_projected, but its
// work space is a file-scope __device__ array that the library reserves when
// it is loaded (every GPU that loads the library holds it until the process
// exits) instead of memory behind a handle.  It reads and writes only the
// caller's device buffers and this array; it allocates nothing.
//
// Sharing: every call uses the same array.  Calls whose kernels may run at the
// same time on the GPU (different streams, or several host threads) race on
// it and must be serialised by the caller.  No entry of the array has to start
// at zero: every value the kernel reads is written earlier in the same call,
// so the contents left by the previous call do no harm.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lslu_internal.cuh"

namespace lslu {
std::string& thread_error();  // defined in lslu_api.cu
}

namespace {

// Largest projected problem the array serves (columns of H).
constexpr int kNoAllocMaxK = 256;
// Work space in doubles: one projected-solve slot for k = 256 (about 133k
// doubles) plus lambda and residual outputs; 1.12 MB.
constexpr int64_t kNoAllocDoubles = 140000;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

__global__ void k_copy_scalars(const double* lam_src, const double* res_src, double* lam_dst,
                               double* res_dst) {
  if (lam_dst) *lam_dst = *lam_src;
  if (res_dst) *res_dst = *res_src;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device (host code only sees a host-side stand-in for the symbol).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

lslu_status fail(lslu_status st, const std::string& msg) {
  lslu::thread_error() = msg;
  return st;
}

}  // namespace

extern "C" lslu_status lslu_projected_noalloc(int32_t k, const double* H, int32_t ldh,
                                              double beta, int32_t rule, double lambda,
                                              int64_t m, double* y, double* sigma, double* c,
                                              double* lambda_out, double* resid_out,
                                              void* cuda_stream) {
  using namespace lslu;
  if (k < 1 || k > kNoAllocMaxK)
    return fail(LSLU_ERR_INVALID_ARG, "lslu_projected_noalloc: k must be in [1, " +
                                          std::to_string(kNoAllocMaxK) + "], got " +
                                          std::to_string(k));
  if (!H || ldh < k + 1) return fail(LSLU_ERR_INVALID_ARG, "lslu_projected_noalloc: invalid H or ldh");
  if (rule < LSLU_LAMBDA_NONE || rule > LSLU_LAMBDA_WGCV || m < 1)
    return fail(LSLU_ERR_INVALID_ARG, "lslu_projected_noalloc: invalid rule or m");
  if (rule == LSLU_LAMBDA_FIXED && !(lambda >= 0.0))
    return fail(LSLU_ERR_INVALID_ARG, "lslu_projected_noalloc: fixed lambda must be >= 0");
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return fail(LSLU_ERR_CUDA, std::string("lslu_projected_noalloc: ") + cudaGetErrorString(e));
  const int CL = projected_cluster_size();
  const int64_t slot = projected_slot_doubles(k, CL);
  if (slot + 2 * kNoAllocMaxK > kNoAllocDoubles)
    return fail(LSLU_ERR_INVALID_ARG, "lslu_projected_noalloc: work space too small for k");
  double* lam_arr = scratch + slot;             // kNoAllocMaxK entries, index k-1
  double* res_arr = lam_arr + kNoAllocMaxK;     // kNoAllocMaxK entries
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  ProjArgs pa = {};
  pa.H = H;
  pa.ldh = ldh;
  pa.beta_val = beta;
  pa.rule = rule;
  pa.lambda = rule == LSLU_LAMBDA_FIXED ? lambda : 0.0;
  pa.m = m;
  pa.k_first = k;
  pa.k_last = k;
  pa.want_y = y != nullptr;
  pa.y = y;
  pa.sig = sigma;
  pa.ldsig = k;
  pa.cvec = c;
  pa.ldc = k + 1;
  pa.lam_out = lam_arr;
  pa.res_out = res_arr;
  ProjWork w;
  w.base = scratch;
  w.cluster = CL;
  e = launch_projected(pa, w, s);
  if (e == cudaSuccess && (lambda_out || resid_out)) {
    k_copy_scalars<<<1, 1, 0, s>>>(lam_arr + (k - 1), res_arr + (k - 1), lambda_out, resid_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return fail(LSLU_ERR_CUDA, std::string("lslu_projected_noalloc: ") + cudaGetErrorString(e));
  return LSLU_OK;
}
