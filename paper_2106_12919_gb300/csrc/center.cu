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
  int64_t N[3];
  int axis;
  int mode;  // 0: nodal -> staggered, 1: staggered -> nodal, 2: bilinear (1/4, 1/2, 1/4) filter
  int m;
  T w[PIC_MAX_CENTER_M];
};

template <class T>
__global__ void stencil_kernel(StencilArgs<T> a) {
  const int64_t ncell = a.N[0] * a.N[1] * a.N[2];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const int64_t iz = e % a.N[2], r = e / a.N[2];
  const int64_t iy = r % a.N[1], ix = r / a.N[1];
  const int64_t idx[3] = {ix, iy, iz};
  const int64_t stride[3] = {a.N[1] * a.N[2], a.N[2], 1};
  const int64_t N = a.N[a.axis], j = idx[a.axis], st = stride[a.axis];
  const int64_t base = e - j * st;
  const int64_t mask = N - 1;
  if (a.mode == 2) {
    // f_j <- f_{j-1} / 4 + f_j / 2 + f_{j+1} / 4 (Sec. 2, the smoothing of the deposits)
    a.out[e] = T(0.25) * a.in[base + ((j - 1) & mask) * st] + T(0.5) * a.in[e] +
               T(0.25) * a.in[base + ((j + 1) & mask) * st];
    return;
  }
  T acc = T(0);
  for (int n = 1; n <= a.m; ++n) {
    int64_t i1, i2;
    if (a.mode == 1) {
      i1 = (j + n - 1) & mask;
      i2 = (j - n) & mask;
    } else {
      i1 = (j + n) & mask;
      i2 = (j - n + 1) & mask;
    }
    acc += a.w[n - 1] * (a.in[base + i1 * st] + a.in[base + i2 * st]);
  }
  a.out[e] = acc;
}

template <class T>
pic_status run(pic_ctx* ctx, const T* in, T* out, int axis, int mode) {
  StencilArgs<T> s;
  memset(&s, 0, sizeof(s));
  s.in = in;
  s.out = out;
  for (int d = 0; d < 3; ++d) s.N[d] = ctx->N[d];
  s.axis = axis;
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
