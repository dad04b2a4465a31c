// FP64 diagnostics: field energy W = 1/2 sum (eps0 |E|^2 + |B|^2 / mu0) dV
// (Sec. 2 (iii)) over a box of cells, and the total of a nodal array.
#include "pic_internal.cuh"

namespace {

template <class T>
struct EnergyArgs {
  const T* F[6];
  int64_t N[3];
  int64_t lo[3], hi[3];
  double* out;  // [2]: sum E^2, sum B^2
};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
__global__ void energy_kernel(EnergyArgs<T> a) {
  const int64_t bx = a.hi[0] - a.lo[0], by = a.hi[1] - a.lo[1], bz = a.hi[2] - a.lo[2];
  const int64_t nb = bx * by * bz;
  double se = 0.0, sb = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t iz = e % bz, r = e / bz;
    const int64_t iy = r % by, ix = r / by;
    const int64_t o = ((a.lo[0] + ix) * a.N[1] + (a.lo[1] + iy)) * a.N[2] + (a.lo[2] + iz);
    for (int c = 0; c < 3; ++c) {
      const double v = (double)a.F[c][o], w = (double)a.F[3 + c][o];
      se += v * v;
      sb += w * w;
    }
  }
  se = block_sum(se);
  sb = block_sum(sb);
  if (threadIdx.x == 0) {
    atomicAdd(a.out, se);
    atomicAdd(a.out + 1, sb);
  }
}

template <class T>
__global__ void sum_kernel(const T* x, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[e];
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

}  // namespace

template <class T>
pic_status diag_energy_t(pic_ctx* ctx, const T* const E[3], const T* const B[3],
                         const int64_t lo[3], const int64_t hi[3], double* out) {
  double* d = reinterpret_cast<double*>(ctx->G);  // scratch: two doubles
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, 2 * sizeof(double), ctx->stream));
  EnergyArgs<T> a;
  for (int c = 0; c < 3; ++c) {
    a.F[c] = E[c];
    a.F[3 + c] = B[c];
    a.N[c] = ctx->N[c];
    a.lo[c] = lo[c];
    a.hi[c] = hi[c];
  }
  a.out = d;
  energy_kernel<T><<<152 * 4, 256, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  double h[2];
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(h, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const double dV = ctx->dx[0] * ctx->dx[1] * ctx->dx[2];
  const double inv_mu0 = ctx->eps0 * ctx->c * ctx->c;
  *out = 0.5 * (ctx->eps0 * h[0] + h[1] * inv_mu0) * dV;
  return PIC_OK;
}

template <class T>
pic_status diag_sum_t(pic_ctx* ctx, const T* a, double* out) {
  double* d = reinterpret_cast<double*>(ctx->G);
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, sizeof(double), ctx->stream));
  sum_kernel<T><<<152 * 4, 256, 0, ctx->stream>>>(a, ctx->ncell, d);
  PIC_LAUNCH_CHECK(ctx);
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

pic_status diag_energy(pic_ctx* ctx, const double* const E[3], const double* const B[3], const int64_t lo[3],
                       const int64_t hi[3], double* out) {
  return diag_energy_t<double>(ctx, E, B, lo, hi, out);
}
pic_status diag_energy32(pic_ctx* ctx, const float* const E[3], const float* const B[3], const int64_t lo[3],
                         const int64_t hi[3], double* out) {
  return diag_energy_t<float>(ctx, E, B, lo, hi, out);
}
pic_status diag_sum(pic_ctx* ctx, const double* a, double* out) { return diag_sum_t<double>(ctx, a, out); }
pic_status diag_sum32(pic_ctx* ctx, const float* a, double* out) { return diag_sum_t<float>(ctx, a, out); }
