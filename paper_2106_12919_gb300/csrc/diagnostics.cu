// Diagnostics the paper uses to compare centering orders and solvers (not on the
// step's hot path): the stencil extent of an update coefficient (Sec. 2 (ii),
// Eq. stencil_extent), the modified wave numbers and centering symbol per axis
// (Sec. 4.1, App. C), the numerical vacuum dispersion of the context's update
// (Sec. 2 (i), App. B) and the averaged transverse RMS size of a beam (Sec. 5.3,
// Eq. RMS_pwfa).  All arithmetic in FP64.
#include "pic_internal.cuh"

#include <cstring>

namespace {

__device__ __forceinline__ double2 z2() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ double2 block_sum2(double2 v) {
  __shared__ double2 red[32];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : z2();
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  return v;
}

// Per index m along `axis` (one block each), sums of the half-spectrum table g over the two
// other Fourier indices, split by the kz plane: P = planes kz = 0 and kz = Nz/2 (self-conjugate),
// Q = the interior planes.  Along z the split is not needed (out[m] = (sum, 0)).
__global__ void extent_reduce_kernel(const double2* g, int64_t Nx, int64_t Ny, int64_t Nz, int axis, double2* PQ) {
  const int64_t nzh = Nz / 2 + 1;
  const int64_t m = blockIdx.x;
  double2 P = z2(), Q = z2();
  if (axis == 2) {
    for (int64_t e = threadIdx.x; e < Nx * Ny; e += blockDim.x) P = add2(P, g[e * nzh + m]);
  } else {
    const int64_t n_other = axis == 0 ? Ny : Nx;
    for (int64_t e = threadIdx.x; e < n_other * nzh; e += blockDim.x) {
      const int64_t kz = e % nzh, o = e / nzh;
      const int64_t ix = axis == 0 ? m : o, iy = axis == 0 ? o : m;
      const double2 v = g[(ix * Ny + iy) * nzh + kz];
      if (kz == 0 || kz == Nz / 2) P = add2(P, v);
      else Q = add2(Q, v);
    }
  }
  P = block_sum2(P);
  Q = block_sum2(Q);
  if (threadIdx.x == 0) {
    PQ[2 * m] = P;
    PQ[2 * m + 1] = Q;
  }
}

// Gamma(x_j) = |(1/Ncell) sum_m F(m) exp(2 pi i m j / N)|, F the sum of g over the full range of
// the two other Fourier indices.  The negative-kz half follows from g(-k) = conj g(k) (g maps real
// fields to real fields):
//   axis x, y: F(m) = P(m) + Q(m) + conj Q(-m);   axis z: F(m) = P(m), F(-m) = conj P(m).
__global__ void extent_dft_kernel(const double2* PQ, int64_t N, int axis, double inv_ncell, double* out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double re = 0.0, im = 0.0;
  for (int64_t m = 0; m < N; ++m) {
    double2 F;
    if (axis == 2) {
      if (m <= N / 2) {
        F = PQ[2 * m];
      } else {
        const double2 p = PQ[2 * (N - m)];
        F = make_double2(p.x, -p.y);
      }
    } else {
      const double2 p = PQ[2 * m], q = PQ[2 * m + 1], qm = PQ[2 * ((N - m) % N) + 1];
      F = make_double2(p.x + q.x + qm.x, p.y + q.y - qm.y);
    }
    double s, c;
    sincospi(2.0 * (double)((m * j) % N) / (double)N, &s, &c);
    re += F.x * c - F.y * s;
    im += F.x * s + F.y * c;
  }
  out[j] = sqrt(re * re + im * im) * inv_ncell;
}

// omega(m) for waves along `axis`: the transverse block of the vacuum update,
// [[TC, -i c^2 TS k], [-i TS k, TC]], has eigenvalues TC +- i c TS k; omega = (largest phase)/dt.
// Along z only m <= Nz/2 is stored: the table at -k is the conjugate, which negates both phases.
__global__ void dispersion_kernel(const double2* TC, const double2* TS, const double* ks, int64_t Ny, int64_t Nz,
                                  int64_t N, int axis, double c, double dt, int fdtd, double* out) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= N) return;
  if (fdtd) {
    // leapfrog: sin(omega dt / 2) = c dt [k]_s / 2 (within the Courant limit checked at creation)
    out[m] = 2.0 * asin(fmin(1.0, 0.5 * c * dt * fabs(ks[m]))) / dt;
    return;
  }
  const int64_t nzh = Nz / 2 + 1;
  const bool mirror = axis == 2 && m > N / 2;
  const int64_t mm = mirror ? N - m : m;
  int64_t mode;
  if (axis == 0) mode = mm * Ny * nzh;
  else if (axis == 1) mode = mm * nzh;
  else mode = mm;
  const double2 tc = TC[mode], ts = TS[mode];
  const double k = ks[mm];
  // TC +- i c TS k
  const double ar = tc.x - c * ts.y * k, ai = tc.y + c * ts.x * k;
  const double br = tc.x + c * ts.y * k, bi = tc.y - c * ts.x * k;
  const double pa = atan2(ai, ar), pb = atan2(bi, br);
  out[m] = (mirror ? -fmin(pa, pb) : fmax(pa, pb)) / dt;
}

// Beam RMS: pass 0 sums w, w x, w y; pass 1 sums w (x - <x>)^2, w (y - <y>)^2 (FP64 sums).
template <class SP>
struct RmsArgs {
  SP sp;
  double dx[2];
  int shz, shy, mask0, mask1;
  const double* mean;  // [3] after pass 0 (sum w, sum w x, sum w y)
  double* acc;
  int pass;
};

template <class SP>
__device__ __forceinline__ void position_xy(const RmsArgs<SP>& a, int64_t p, double& x, double& y);

template <>
__device__ __forceinline__ void position_xy<pic_species>(const RmsArgs<pic_species>& a, int64_t p, double& x,
                                                         double& y) {
  x = a.sp.x[p];
  y = a.sp.y[p];
}

template <>
__device__ __forceinline__ void position_xy<pic_species32>(const RmsArgs<pic_species32>& a, int64_t p, double& x,
                                                           double& y) {
  const int c = a.sp.cell[p];
  const int ix = (c >> (a.shz + a.shy)) & a.mask0, iy = (c >> a.shz) & a.mask1;
  x = ((double)ix + (double)a.sp.fx[p]) * a.dx[0];
  y = ((double)iy + (double)a.sp.fy[p]) * a.dx[1];
}

template <class SP, class W>
__global__ void rms_kernel(RmsArgs<SP> a, const W* w) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  double mx = 0.0, my = 0.0;
  if (a.pass == 1) {
    mx = a.mean[1] / a.mean[0];
    my = a.mean[2] / a.mean[0];
  }
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.sp.n; p += (int64_t)gridDim.x * blockDim.x) {
    double x, y;
    position_xy<SP>(a, p, x, y);
    const double wp = (double)w[p];
    if (a.pass == 0) {
      s0 += wp;
      s1 += wp * x;
      s2 += wp * y;
    } else {
      s1 += wp * (x - mx) * (x - mx);
      s2 += wp * (y - my) * (y - my);
    }
  }
  double2 r = block_sum2(make_double2(s0, s1));
  double2 t = block_sum2(make_double2(s2, 0.0));
  if (threadIdx.x == 0) {
    atomicAdd(a.acc, r.x);
    atomicAdd(a.acc + 1, r.y);
    atomicAdd(a.acc + 2, t.x);
  }
}

int ilog2i(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

template <class SP, class W>
pic_status beam_rms(pic_ctx* ctx, const SP* sp, const W* w, double* delta) {
  if (!sp || !delta) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  if (sp->n <= 0) return pic_set_error(ctx, PIC_ERR_ARG, "empty species");
  double* d = reinterpret_cast<double*>(ctx->G);  // scratch: [3] pass-0 sums, [3] pass-1 sums
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, 6 * sizeof(double), ctx->stream));
  RmsArgs<SP> a;
  a.sp = *sp;
  a.dx[0] = ctx->dx[0];
  a.dx[1] = ctx->dx[1];
  a.shz = ilog2i(ctx->N[2]);
  a.shy = ilog2i(ctx->N[1]);
  a.mask0 = (int)ctx->N[0] - 1;
  a.mask1 = (int)ctx->N[1] - 1;
  a.mean = d;
  for (int pass = 0; pass < 2; ++pass) {
    a.pass = pass;
    a.acc = d + 3 * pass;
    rms_kernel<SP, W><<<152 * 4, 256, 0, ctx->stream>>>(a, w);
    PIC_LAUNCH_CHECK(ctx);
  }
  double h[6];
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(h, d, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (!(h[0] > 0.0)) return pic_set_error(ctx, PIC_ERR_ARG, "sum of weights is not positive");
  *delta = 0.5 * sqrt(h[4] / h[0]) + 0.5 * sqrt(h[5] / h[0]);
  return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_stencil_extent(pic_ctx* ctx, const char* coef, int axis, double* out) {
  if (!ctx) return PIC_ERR_ARG;
  if (!coef || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  if (axis < 0 || axis > 2) return pic_set_error(ctx, PIC_ERR_ARG, "axis must be 0, 1 or 2");
  const int k = coef_index(ctx, coef);
  if (k < 0) return pic_set_error(ctx, PIC_ERR_ARG, "unknown coefficient '%s'", coef);
  const int64_t N = ctx->N[axis];
  const int64_t nred = axis == 2 ? ctx->nzh : N;
  double2* PQ = reinterpret_cast<double2*>(ctx->G);  // scratch: 2 nred double2, then N doubles
  double* g = reinterpret_cast<double*>(PQ + 2 * nred);
  extent_reduce_kernel<<<(unsigned)nred, 256, 0, ctx->stream>>>(ctx->coef + k * ctx->nmode, ctx->N[0], ctx->N[1],
                                                                ctx->N[2], axis, PQ);
  PIC_LAUNCH_CHECK(ctx);
  extent_dft_kernel<<<(unsigned)((N + 127) / 128), 128, 0, ctx->stream>>>(PQ, N, axis, 1.0 / (double)ctx->ncell, g);
  PIC_LAUNCH_CHECK(ctx);
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(out, g, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

pic_status pic_axis_tables(pic_ctx* ctx, int axis, double* ks, double* kc, double* zeta) {
  if (!ctx) return PIC_ERR_ARG;
  if (axis < 0 || axis > 2) return pic_set_error(ctx, PIC_ERR_ARG, "axis must be 0, 1 or 2");
  const size_t bytes = ctx->N[axis] * sizeof(double);
  const double* src[3] = {ctx->ks[axis], ctx->kc[axis], ctx->zeta[axis]};
  double* dst[3] = {ks, kc, zeta};
  for (int t = 0; t < 3; ++t)
    if (dst[t]) PIC_CUDA_TRY(ctx, cudaMemcpyAsync(dst[t], src[t], bytes, cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

pic_status pic_vacuum_dispersion(pic_ctx* ctx, int axis, double* omega) {
  if (!ctx) return PIC_ERR_ARG;
  if (!omega) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  if (axis < 0 || axis > 2) return pic_set_error(ctx, PIC_ERR_ARG, "axis must be 0, 1 or 2");
  const int64_t N = ctx->N[axis];
  double* d = reinterpret_cast<double*>(ctx->G);
  dispersion_kernel<<<(unsigned)((N + 127) / 128), 128, 0, ctx->stream>>>(
      ctx->coef + COEF_TC * ctx->nmode, ctx->coef + COEF_TS * ctx->nmode, ctx->ks[axis], ctx->N[1], ctx->N[2], N,
      axis, ctx->c, ctx->dt, ctx->cycle == PIC_CYCLE_HYBRID_FDTD ? 1 : 0, d);
  PIC_LAUNCH_CHECK(ctx);
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(omega, d, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

pic_status pic_beam_rms(pic_ctx* ctx, const pic_species* sp, double* delta) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!sp) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  if (!sp->x || !sp->y || !sp->w) return pic_set_error(ctx, PIC_ERR_ARG, "null particle array");
  return beam_rms<pic_species, double>(ctx, sp, sp->w, delta);
}

pic_status pic_beam_rms32(pic_ctx* ctx, const pic_species32* sp, double* delta) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP32) return pic_set_error(ctx, PIC_ERR_ARG, "FP32 entry point on an FP64 context");
  if (!sp) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  if (!sp->cell || !sp->fx || !sp->fy || !sp->w) return pic_set_error(ctx, PIC_ERR_ARG, "null particle array");
  return beam_rms<pic_species32, float>(ctx, sp, sp->w, delta);
}

}  // extern "C"
