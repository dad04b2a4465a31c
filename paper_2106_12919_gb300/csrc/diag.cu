// FP64 diagnostics: field energy W = 1/2 sum (eps0 |E|^2 + |B|^2 / mu0) dV
// (Sec. 2 (iii)) over a box of cells, and the total of a nodal array.
#include "pic_internal.cuh"

namespace {

template <class T>
struct EnergyArgs {
  const T* F[6];
  int64_t N[3];
  int64_t lo[3], hi[3];
  int contiguous;  // the box spans whole y-z planes
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

// Vector of four consecutive elements (16 B for FP32, 32 B as two 16 B loads for FP64).
__device__ __forceinline__ void load4(const float* p, double* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Running sum s + c of squares in two FP32 words (Knuth's TwoSum for the running sum, the exact
// square v^2 = p + e from one FMA): the pair carries ~48 bits, so FP32 data is summed to FP64-grade
// accuracy at FP32 rate (this part's FP64 units would bound the kernel: ~0.3 ms for 50M squares).
struct SumF2 {
  float s = 0.0f, c = 0.0f;
  // explicit round-to-nearest operations: the compiler must not fuse s + v * v into one FMA
  __device__ __forceinline__ void add_sq(float v) {
    const float p = __fmul_rn(v, v);
    const float e = fmaf(v, v, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    c = __fadd_rn(c, __fadd_rn(err, e));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Sums of |E|^2 and |B|^2 over the box: FP64 data in FP64, FP32 data in two-float pairs per thread
// and FP64 across threads.  The box
// is walked in z-rows: with the row start and length multiples of 4 (vec4) each thread takes
// four consecutive elements of all six components per iteration; otherwise one element.
template <class T, bool VEC>
__global__ void energy_kernel(EnergyArgs<T> a) {
  const int64_t by = a.hi[1] - a.lo[1], bz = a.hi[2] - a.lo[2];
  const int64_t nrow = (a.hi[0] - a.lo[0]) * by;
  const int64_t per_row = VEC ? bz / 4 : bz;
  const int64_t total = nrow * per_row;
  double se[3] = {0.0, 0.0, 0.0}, sb[3] = {0.0, 0.0, 0.0};
  SumF2 fe[3], fb[3];
  constexpr bool F32 = sizeof(T) == 4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t o;
    if (a.contiguous) {  // full y-z planes: the box is one contiguous range
      o = a.lo[0] * a.N[1] * a.N[2] + (VEC ? 4 * e : e);
    } else {
      const int64_t r = e / per_row, iz = e - r * per_row;
      const int64_t ix = r / by, iy = r - ix * by;
      o = ((a.lo[0] + ix) * a.N[1] + (a.lo[1] + iy)) * a.N[2] + a.lo[2] + (VEC ? 4 * iz : iz);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (F32 && VEC) {
        const float4 v = *reinterpret_cast<const float4*>(a.F[c] + o);
        const float4 w = *reinterpret_cast<const float4*>(a.F[3 + c] + o);
        fe[c].add_sq(v.x);
        fe[c].add_sq(v.y);
        fe[c].add_sq(v.z);
        fe[c].add_sq(v.w);
        fb[c].add_sq(w.x);
        fb[c].add_sq(w.y);
        fb[c].add_sq(w.z);
        fb[c].add_sq(w.w);
      } else if (F32) {
        fe[c].add_sq((float)a.F[c][o]);
        fb[c].add_sq((float)a.F[3 + c][o]);
      } else if (VEC) {
        double v[4], w[4];
        load4(a.F[c] + o, v);
        load4(a.F[3 + c] + o, w);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          se[c] = fma(v[k], v[k], se[c]);
          sb[c] = fma(w[k], w[k], sb[c]);
        }
      } else {
        const double v = (double)a.F[c][o], w = (double)a.F[3 + c][o];
        se[c] = fma(v, v, se[c]);
        sb[c] = fma(w, w, sb[c]);
      }
    }
  }
  if (F32)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      se[c] = fe[c].value();
      sb[c] = fb[c].value();
    }
  double te = block_sum(se[0] + se[1] + se[2]);
  double tb = block_sum(sb[0] + sb[1] + sb[2]);
  if (threadIdx.x == 0) {
    atomicAdd(a.out, te);
    atomicAdd(a.out + 1, tb);
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
  a.contiguous = lo[1] == 0 && hi[1] == ctx->N[1] && lo[2] == 0 && hi[2] == ctx->N[2];
  // vector path: rows start and end on 4-element boundaries (the arrays are cudaMalloc-aligned)
  bool vec = (lo[2] % 4 == 0) && (hi[2] % 4 == 0) && (ctx->N[2] % 4 == 0);
  for (int c = 0; c < 6; ++c) vec = vec && (reinterpret_cast<uintptr_t>(a.F[c]) % (4 * sizeof(T)) == 0);
  if (vec)
    energy_kernel<T, true><<<152 * 16, 256, 0, ctx->stream>>>(a);
  else
    energy_kernel<T, false><<<152 * 16, 256, 0, ctx->stream>>>(a);
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
