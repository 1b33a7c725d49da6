// Box solve that allocates nothing: the padded work grid and the transform
// tables live in one file-scope device array instead of cudaMalloc'd
// workspace.  Meant for callers that must not allocate device memory
// themselves or through a library (for example code running inside a memory
// pool or arena that owns all of the device memory, or under a policy that
// forbids allocation after start-up).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace kfbi {
namespace {

constexpr int NA_MAX_N = 512;
constexpr size_t NA_TABLE = NA_MAX_N + 4 * NA_MAX_N;  // mu[N] and twiddles e^{i pi j/N}, j < 2N
constexpr size_t NA_TOTAL = (size_t)KFBI_NOALLOC_MAX_POINTS + NA_TABLE;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (looked up once
// per device with that device current)
int scratch_address(double** out) {
  int dev = 0;
  KFBI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("device index %d out of range", dev);
    return KFBI_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    KFBI_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return KFBI_OK;
}

// mu1[k] = -(4/h^2) sin^2(pi k / (2N)) and e^{i pi j / N} on the device
__global__ void k_noalloc_tables(double* mu, double* tw, int N, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const double s = sinpi((double)i / (2.0 * N));
    mu[i] = -(4.0 / (h * h)) * s * s;
  }
  if (i < 2 * N) {
    double sv, cv;
    sincospi((double)i / (double)N, &sv, &cv);
    tw[2 * i] = cv;
    tw[2 * i + 1] = sv;
  }
}

}  // namespace
}  // namespace kfbi

extern "C" int kfbi_box_solve_noalloc(int dim, int N, double lo, double hi, double lambda, const double* r_dev,
                                      double* v_dev, void* stream) {
  using namespace kfbi;
  if ((dim != 2 && dim != 3) || !dst_supported(N) || !(hi > lo) || r_dev == nullptr || v_dev == nullptr) {
    set_error("kfbi_box_solve_noalloc: bad arguments (dim 2 or 3, N in 8..512, hi > lo, non-null fields)");
    return KFBI_ERR_ARG;
  }
  const size_t points = dim == 3 ? (size_t)N * N * N : (size_t)N * N;
  if (points > (size_t)KFBI_NOALLOC_MAX_POINTS) {
    set_error("kfbi_box_solve_noalloc: N^dim = %zu exceeds the static scratch of %d points "
              "(3-D N <= 64, 2-D N <= 512)", points, KFBI_NOALLOC_MAX_POINTS);
    return KFBI_ERR_ARG;
  }
  double* base = nullptr;
  if (int rc = scratch_address(&base)) return rc;
  double* work = base;
  double* mu = base + KFBI_NOALLOC_MAX_POINTS;
  double* tw = mu + NA_MAX_N;
  cudaStream_t st = (cudaStream_t)stream;
  // a handle on the stack that only carries the grid, stream and tables
  kfbi_handle tmp;
  tmp.grid.dim = dim;
  tmp.grid.N = N;
  tmp.grid.lo = lo;
  tmp.grid.h = (hi - lo) / N;
  tmp.stream = st;
  tmp.t.mu = mu;
  tmp.t.tw64 = tw;
  k_noalloc_tables<<<(2 * N + 127) / 128, 128, 0, st>>>(mu, tw, N, tmp.grid.h);
  KFBI_CHECK_LAUNCH();
  // the passes never write the z = 0 plane of the padded 3-D grid: it must
  // hold the zero boundary value whatever the previous call left there
  if (dim == 3) KFBI_CUDA(cudaMemsetAsync(work, 0, sizeof(double) * (size_t)N * N, st));
  SolveArgs sa;
  sa.src = r_dev;
  sa.lambda = lambda;
  sa.out_user = v_dev;
  return box_solve64(&tmp, sa, work);
}
