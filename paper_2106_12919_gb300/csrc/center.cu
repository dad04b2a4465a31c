// Finite-order centering between the nodal and Yee grids as real-space stencils
// (Sec. 3, Eq. staggered_finite_sum, periodic).  pic_step applies the same
// operators as their Fourier symbol inside the k-space update; these kernels
// are the stand-alone form of the two centering rows of the step, and the
// centering of the FDTD cycle (FP64 and FP32), which also filters its J here.
//
// staggered -> nodal along axis a: f_j = sum_n w_n (s[j+n-1] + s[j-n]),
// nodal -> staggered:               f_{j+1/2} = sum_n w_n (g[j+n] + g[j-n+1]),
// with w_n = alpha^s_{m,n} / 2 and s[i] the value at (i + 1/2) dx.
#include "pic_internal.cuh"

namespace {

template <class T>
struct StencilArgs {
  const T* in;
  T* out;
  int ncell;
  int shift, mask;  // the axis: index stride 2^shift, coordinate j = (e >> shift) & mask
  int mode;  // 0: nodal -> staggered, 1: staggered -> nodal, 2: bilinear (1/4, 1/2, 1/4) filter
  int m;
  T w[PIC_MAX_CENTER_M];
};

// One output element per thread; grids are powers of two (at most 2^30 cells), so the index
// arithmetic is 32-bit shifts and masks.
template <class T>
__global__ void __launch_bounds__(256) stencil_kernel(StencilArgs<T> a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ncell) return;
  const int j = (e >> a.shift) & a.mask;
  const int base = e - (j << a.shift);
  const T* in = a.in;
  if (a.mode == 2) {
    // f_j <- f_{j-1} / 4 + f_j / 2 + f_{j+1} / 4 (Sec. 2, the smoothing of the deposits)
    a.out[e] = T(0.25) * in[base + (((j - 1) & a.mask) << a.shift)] + T(0.5) * in[e] +
               T(0.25) * in[base + (((j + 1) & a.mask) << a.shift)];
    return;
  }
  // mode 1: f_j = sum_n w_n (s[j+n-1] + s[j-n]); mode 0: f_{j+1/2} = sum_n w_n (g[j+n] + g[j-n+1])
  const int d = a.mode == 1 ? -1 : 0;
  T acc = T(0);
#pragma unroll
  for (int n = 1; n <= PIC_MAX_CENTER_M; ++n) {
    if (n > a.m) break;
    const int i1 = (j + n + d) & a.mask, i2 = (j - n + 1 + d) & a.mask;
    acc += a.w[n - 1] * (in[base + (i1 << a.shift)] + in[base + (i2 << a.shift)]);
  }
  a.out[e] = acc;
}

int lg2i(int64_t n) {
  int s = 0;
  while ((int64_t(1) << s) < n) ++s;
  return s;
}

template <class T>
pic_status run(pic_ctx* ctx, const T* in, T* out, int axis, int mode) {
  StencilArgs<T> s;
  memset(&s, 0, sizeof(s));
  s.in = in;
  s.out = out;
  s.ncell = (int)ctx->ncell;
  s.shift = axis == 0 ? lg2i(ctx->N[1]) + lg2i(ctx->N[2]) : axis == 1 ? lg2i(ctx->N[2]) : 0;
  s.mask = (int)ctx->N[axis] - 1;
  s.mode = mode;
  s.m = ctx->cw[axis].m;
  for (int n = 0; n < s.m; ++n) s.w[n] = (T)ctx->cw[axis].w[n];
  const int bs = 256;
  stencil_kernel<T><<<(unsigned)((ctx->ncell + bs - 1) / bs), bs, 0, ctx->stream>>>(s);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

// staggered axes of E^x..B^z as bit masks (x = 1, y = 2, z = 4)
const int kStag[6] = {1, 2, 4, 2 | 4, 1 | 4, 1 | 2};

// Apply the stencils of every axis in mask (x, y, z order) from in to out,
// using two work arrays for the intermediate results.
template <class T>
pic_status apply(pic_ctx* ctx, const T* in, T* out, int mask, int mode, T* w0, T* w1) {
  int axes[3], na = 0;
  for (int a = 0; a < 3; ++a)
    if (mask & (1 << a)) axes[na++] = a;
  const T* src = in;
  for (int q = 0; q < na; ++q) {
    T* dst = (q == na - 1) ? out : (q % 2 == 0 ? w0 : w1);
    PIC_TRY(run<T>(ctx, src, dst, axes[q], mode));
    src = dst;
  }
  return PIC_OK;
}

}  // namespace

template <class T>
pic_status center_to_nodal_t(pic_ctx* ctx, const T* const F[6], T* const out[6], T* w0, T* w1) {
  for (int c = 0; c < 6; ++c) PIC_TRY(apply<T>(ctx, F[c], out[c], kStag[c], 1, w0, w1));
  return PIC_OK;
}

template <class T>
pic_status center_to_yee_t(pic_ctx* ctx, const T* const Jn[3], T* const out[3], T* w0, T* w1) {
  for (int c = 0; c < 3; ++c) PIC_TRY(apply<T>(ctx, Jn[c], out[c], kStag[c], 0, w0, w1));
  return PIC_OK;
}

template <class T>
pic_status bilinear_filter_t(pic_ctx* ctx, T* f, int passes, T* w0, T* w1) {
  for (int p = 0; p < passes; ++p) {
    PIC_TRY(run<T>(ctx, f, w0, 0, 2));
    PIC_TRY(run<T>(ctx, w0, w1, 1, 2));
    PIC_TRY(run<T>(ctx, w1, f, 2, 2));
  }
  return PIC_OK;
}

template pic_status center_to_nodal_t<double>(pic_ctx*, const double* const[6], double* const[6], double*, double*);
template pic_status center_to_nodal_t<float>(pic_ctx*, const float* const[6], float* const[6], float*, float*);
template pic_status center_to_yee_t<double>(pic_ctx*, const double* const[3], double* const[3], double*, double*);
template pic_status center_to_yee_t<float>(pic_ctx*, const float* const[3], float* const[3], float*, float*);
template pic_status bilinear_filter_t<double>(pic_ctx*, double*, int, double*, double*);
template pic_status bilinear_filter_t<float>(pic_ctx*, float*, int, float*, float*);

pic_status center_to_nodal(pic_ctx* ctx, const double* const F[6], double* const out[6]) {
  return center_to_nodal_t<double>(ctx, F, out, ctx->Jn, ctx->Jn + ctx->ncell);
}

pic_status center_to_yee(pic_ctx* ctx, const double* const Jn[3], double* const out[3]) {
  return center_to_yee_t<double>(ctx, Jn, out, ctx->nodal, ctx->nodal + ctx->ncell);
}
