// Allocation-free variant of the Yee -> nodal centering (pic_center_to_nodal_static).
//
// pic_center_to_nodal needs a pic_ctx, and pic_init allocates device memory.
// This entry point needs neither: its only scratch (the intermediate result of
// the two-axis centering of B) lives in a file-scope static device array that
// the CUDA runtime reserves on every device that loads the library, until the
// process exits.  It never calls cudaMalloc, cudaFree or any allocating library.
#include "pic_internal.cuh"

#include <cmath>
#include <mutex>

namespace {

// 2^21 doubles = 16 MiB: grids up to 2,097,152 cells (e.g. 128 x 128 x 128).
constexpr int64_t kStaticScratchCells = int64_t(1) << 21;
static __device__ __align__(256) double g_center_scratch[kStaticScratchCells];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};  // device address of g_center_scratch, per device

struct StaticStencilArgs {
  const double* in;
  double* out;
  int64_t N[3];
  int axis;
  CenterWeights cw;
};

// f_j = sum_n w_n (s[j+n-1] + s[j-n]) along `axis`, periodic (Sec. 3, Eq. staggered_finite_sum).
__global__ void static_stencil_kernel(StaticStencilArgs a) {
  const int64_t ncell = a.N[0] * a.N[1] * a.N[2];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const int64_t iz = e % a.N[2], r = e / a.N[2];
  const int64_t iy = r % a.N[1], ix = r / a.N[1];
  const int64_t idx[3] = {ix, iy, iz};
  const int64_t stride[3] = {a.N[1] * a.N[2], a.N[2], 1};
  const int64_t N = a.N[a.axis], j = idx[a.axis], st = stride[a.axis];
  const int64_t base = e - j * st, mask = N - 1;
  double acc = 0.0;
  for (int n = 1; n <= a.cw.m; ++n)
    acc += a.cw.w[n - 1] * (a.in[base + ((j + n - 1) & mask) * st] + a.in[base + ((j - n) & mask) * st]);
  a.out[e] = acc;
}

// alpha^s_{m,n} / 2 (Eq. eq_Fornberg_staggered), in long double then rounded.
void center_weights(int order, CenterWeights* cw) {
  const int m = order / 2;
  long double dfact = 1.0L;
  for (int i = 1; i <= m; ++i) dfact *= (2.0L * i - 1.0L) / 2.0L;
  cw->m = m;
  for (int n = 1; n <= m; ++n) {
    long double f1 = 1.0L, f2 = 1.0L;
    for (int i = 2; i <= m - n; ++i) f1 *= i;
    for (int i = 2; i <= m + n - 1; ++i) f2 *= i;
    const long double a = ((n % 2) ? 1.0L : -1.0L) * dfact * dfact * 4.0L / ((2.0L * n - 1.0L) * f1 * f2);
    cw->w[n - 1] = (double)(a / 2.0L);
  }
}

// Device address of the static scratch on the current device; looked up once per device.
pic_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    fprintf(stderr, "pic_center_to_nodal_static: no usable current CUDA device\n");
    return PIC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_center_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fprintf(stderr, "pic_center_to_nodal_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return PIC_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_center_to_nodal_static(const int64_t grid[3], const int32_t centering_order[3],
                                                 const double* const F[6], double* const out[6],
                                                 void* cuda_stream) {
  if (!grid || !centering_order || !F || !out) return PIC_ERR_ARG;
  for (int c = 0; c < 6; ++c)
    if (!F[c] || !out[c]) return PIC_ERR_ARG;
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    const int64_t n = grid[a];
    const int co = centering_order[a];
    if (n < 2 || n > 1024 || (n & (n - 1)) != 0) return PIC_ERR_UNSUPPORTED;
    if (co < 2 || co % 2 || co / 2 > PIC_MAX_CENTER_M || co > n) return PIC_ERR_ARG;
    ncell *= n;
  }
  if (ncell > kStaticScratchCells) {
    fprintf(stderr, "pic_center_to_nodal_static: %lld cells exceed the static scratch maximum of %lld cells\n",
            (long long)ncell, (long long)kStaticScratchCells);
    return PIC_ERR_CAPACITY;
  }
  if (arrays_overlap(reinterpret_cast<const void* const*>(F), 6, reinterpret_cast<const void* const*>(out), 6,
                     (size_t)ncell * sizeof(double)))
    return PIC_ERR_ARG;  // stencil passes cannot run in place
  double* scratch = nullptr;
  const pic_status st = scratch_address(&scratch);
  if (st != PIC_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  static const int kStag[6] = {1, 2, 4, 2 | 4, 1 | 4, 1 | 2};  // staggered axes of Ex..Bz
  StaticStencilArgs s;
  for (int a = 0; a < 3; ++a) s.N[a] = grid[a];
  const int bs = 256;
  const unsigned nb = (unsigned)((ncell + bs - 1) / bs);
  for (int c = 0; c < 6; ++c) {
    int axes[3], na = 0;
    for (int a = 0; a < 3; ++a)
      if (kStag[c] & (1 << a)) axes[na++] = a;
    const double* src = F[c];
    for (int q = 0; q < na; ++q) {
      s.in = src;
      s.out = (q == na - 1) ? out[c] : scratch;  // first of two passes goes through the scratch
      s.axis = axes[q];
      center_weights(centering_order[axes[q]], &s.cw);
      static_stencil_kernel<<<nb, bs, 0, stream>>>(s);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        fprintf(stderr, "pic_center_to_nodal_static: launch failed: %s\n", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
      }
      src = s.out;
    }
  }
  return PIC_OK;
}
