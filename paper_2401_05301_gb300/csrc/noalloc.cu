// Allocation-free variant of the nearest-neighbour correlator of one bond.
//
// The handle-based path (tebd_measure) computes C_j = <b+_j b_{j+1}> for every
// bond with scratch buffers that the library allocates.  Some callers cannot
// allocate device memory at the point where they need this number: code that
// runs under a fixed device-memory budget, code inside a framework whose
// allocator must own every device byte, and latency-critical loops where a
// cudaMalloc would synchronise the device.  tebd_bond_correlator_noalloc
// serves them: the caller passes device inputs and a device output, and the
// scratch lives in a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (1,179,648 bytes), which every GPU that loads the library holds until the
// process exits.
#include "ptebd.h"
#include "ptebd_internal.h"

#include <cstdio>

using namespace ptebd;

namespace {

constexpr int NA_MAX_CHI = 64;  // largest chi_l, chi_m, chi_r accepted
constexpr int NA_MAX_D = 8;     // largest local dimension accepted (n_max <= 7)
constexpr size_t NA_BIG = (size_t)NA_MAX_CHI * NA_MAX_D * NA_MAX_CHI;  // P' and Q' (complex elements)
constexpr size_t NA_SMALL = (size_t)NA_MAX_CHI * NA_MAX_CHI;           // X and Y^T
constexpr size_t NA_TOTAL = 2 * NA_BIG + 2 * NA_SMALL;
constexpr size_t NOALLOC_SCRATCH_BYTES = NA_TOTAL * sizeof(double2);

// Shared by every call on a device; calls that overlap on the GPU race on it.
static __device__ __align__(256) double2 g_noalloc_scratch[NA_TOTAL];
static_assert(sizeof(g_noalloc_scratch) == NOALLOC_SCRATCH_BYTES, "scratch size");
static_assert(NOALLOC_SCRATCH_BYTES == 1179648, "the documented scratch size");

// Device address of the scratch array in the context current on the calling
// thread.  The host-side symbol g_noalloc_scratch is only a stand-in: a kernel
// must be given the address cudaGetSymbolAddress returns with the device
// current.  The address is looked up on every call rather than cached per
// device ordinal: after cudaDeviceReset, or with another context current on
// the same device, the library's device code is loaded again at a different
// address, and a cached pointer would then point at memory this call does
// not own.  The first lookup in a context loads the module there.
int scratch_in_current_context(double2** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();  // no error was pending on entry, so this clears only our own
    return TEBD_ERR_CUDA;
  }
  *out = static_cast<double2*>(p);
  return TEBD_OK;
}

}  // namespace

extern "C" int tebd_bond_correlator_noalloc(const double* B_left, const double* lam_left, const double* B_right,
                                             int chi_l, int chi_m, int chi_r, int d, double* C_out,
                                             void* cuda_stream) {
  if (!B_left || !lam_left || !B_right || !C_out) return TEBD_ERR_ARG;
  if (chi_l < 1 || chi_m < 1 || chi_r < 1 || d < 2) return TEBD_ERR_ARG;
  if (chi_l > NA_MAX_CHI || chi_m > NA_MAX_CHI || chi_r > NA_MAX_CHI || d > NA_MAX_D) {
    std::fprintf(stderr,
                 "tebd_bond_correlator_noalloc: chi_l=%d chi_m=%d chi_r=%d d=%d exceeds the fixed scratch "
                 "(chi <= %d, d <= %d)\n",
                 chi_l, chi_m, chi_r, d, NA_MAX_CHI, NA_MAX_D);
    return TEBD_ERR_TOO_LARGE;
  }
  // An error left pending by earlier work (another library, or a kernel that
  // faulted) belongs to its owner: report it without clearing it and launch nothing.
  if (cudaPeekAtLastError() != cudaSuccess) return TEBD_ERR_CUDA;
  double2* scratch = nullptr;
  if (int r = scratch_in_current_context(&scratch)) return r;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const double2* Bl = reinterpret_cast<const double2*>(B_left);
  const double2* Br = reinterpret_cast<const double2*>(B_right);
  // Every scratch element read below is first written by this call, so the
  // contents left by an earlier call never leak into the result.
  double2* P = scratch;                       // [chi_l * d][chi_m]
  double2* Q = scratch + NA_BIG;              // [chi_m][d * chi_r]
  double2* X = scratch + 2 * NA_BIG;          // [chi_m][chi_m]
  double2* Yt = scratch + 2 * NA_BIG + NA_SMALL;
  launch_shift_left(Bl, lam_left, P, chi_l, d, chi_m, s);
  launch_shift_right(Br, Q, chi_m, d, chi_r, s);
  GemmProb px{};
  px.A = P; px.B = Bl; px.C = X;
  px.lda = chi_m; px.ldb = chi_m; px.ldc = chi_m;
  px.M = chi_m; px.N = chi_m; px.K = chi_l * d; px.batch = 1;
  px.red_div = px.row_div = px.col_div = 1;
  px.alpha_re = 1.0;
  gemm_launch_single(true, OP_C, OP_N, px, s);
  GemmProb py = px;
  py.A = Q; py.B = Br; py.C = Yt;
  py.lda = (long long)d * chi_r; py.ldb = (long long)d * chi_r; py.ldc = chi_m;
  py.K = d * chi_r;
  gemm_launch_single(true, OP_N, OP_C, py, s);
  launch_trace_product(X, Yt, chi_m, reinterpret_cast<double2*>(C_out), s);
  // only this call's launches can have set the error read here
  if (cudaGetLastError() != cudaSuccess) return TEBD_ERR_CUDA;
  return TEBD_OK;
}
