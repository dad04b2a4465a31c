// Finite-order centering between the nodal and Yee grids as real-space stencils
// (Sec. 3, Eq. staggered_finite_sum, periodic).  pic_step applies the same
// operators as their Fourier symbol inside the k-space update; these kernels
// are the stand-alone form of the two centering rows of the step.
//
// staggered -> nodal along axis a: f_j = sum_n w_n (s[j+n-1] + s[j-n]),
// nodal -> staggered:               f_{j+1/2} = sum_n w_n (g[j+n] + g[j-n+1]),
// with w_n = alpha^s_{m,n} / 2 and s[i] the value at (i + 1/2) dx.
#include "pic_internal.cuh"

namespace {

struct StencilArgs {
  const double* in;
  double* out;
  int64_t N[3];
  int axis;
  int to_nodal;
  CenterWeights cw;
};

__global__ void stencil_kernel(StencilArgs a) {
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
  double acc = 0.0;
  for (int n = 1; n <= a.cw.m; ++n) {
    int64_t i1, i2;
    if (a.to_nodal) {
      i1 = (j + n - 1) & mask;
      i2 = (j - n) & mask;
    } else {
      i1 = (j + n) & mask;
      i2 = (j - n + 1) & mask;
    }
    acc += a.cw.w[n - 1] * (a.in[base + i1 * st] + a.in[base + i2 * st]);
  }
  a.out[e] = acc;
}

pic_status run(pic_ctx* ctx, const double* in, double* out, int axis, int to_nodal) {
  StencilArgs s;
  s.in = in;
  s.out = out;
  for (int d = 0; d < 3; ++d) s.N[d] = ctx->N[d];
  s.axis = axis;
  s.to_nodal = to_nodal;
  s.cw = ctx->cw[axis];
  const int bs = 256;
  stencil_kernel<<<(unsigned)((ctx->ncell + bs - 1) / bs), bs, 0, ctx->stream>>>(s);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

// staggered axes of E^x..B^z as bit masks (x = 1, y = 2, z = 4)
const int kStag[6] = {1, 2, 4, 2 | 4, 1 | 4, 1 | 2};

// Apply the stencils of every axis in mask (x, y, z order) from in to out,
// using two work arrays for the intermediate results.
pic_status apply(pic_ctx* ctx, const double* in, double* out, int mask, int to_nodal, double* w0,
                 double* w1) {
  int axes[3], na = 0;
  for (int a = 0; a < 3; ++a)
    if (mask & (1 << a)) axes[na++] = a;
  const double* src = in;
  for (int q = 0; q < na; ++q) {
    double* dst = (q == na - 1) ? out : (q % 2 == 0 ? w0 : w1);
    pic_status st = run(ctx, src, dst, axes[q], to_nodal);
    if (st != PIC_OK) return st;
    src = dst;
  }
  return PIC_OK;
}

}  // namespace

pic_status center_to_nodal(pic_ctx* ctx, const double* const F[6], double* const out[6]) {
  for (int c = 0; c < 6; ++c) {
    pic_status st = apply(ctx, F[c], out[c], kStag[c], 1, ctx->Jn, ctx->Jn + ctx->ncell);
    if (st != PIC_OK) return st;
  }
  return PIC_OK;
}

pic_status center_to_yee(pic_ctx* ctx, const double* const Jn[3], double* const out[3]) {
  for (int c = 0; c < 3; ++c) {
    pic_status st = apply(ctx, Jn[c], out[c], kStag[c], 0, ctx->nodal, ctx->nodal + ctx->ncell);
    if (st != PIC_OK) return st;
  }
  return PIC_OK;
}
