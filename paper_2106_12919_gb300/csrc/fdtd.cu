// The hybrid scheme with a finite-difference (FDTD) field solver: the adaptation to FDTD the
// conclusions (Sec. 6) state.  Particles gather from and deposit to the nodes as in the hybrid
// PSATD cycle, the finite-order centering of Sec. 3 (Eq. staggered_finite_sum) moves E, B to the
// nodes and J to the Yee grid in real space, and the Yee-grid fields advance by leapfrog with
// the B update split in halves so that E and B are both known at integer times:
//
//   B^{n+1/2} = B^n - (dt/2) curl E^n
//   E^{n+1}   = E^n + dt (c^2 curl B^{n+1/2} - J^{n+1/2} / eps0)
//   B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1}
//
// Each derivative is the staggered difference of order 2m along its axis,
//   (D f)_{j+1/2} = sum_{n=1}^{m} c_n (f_{j+n} - f_{j-n+1}) / dx,  c_n = alpha^s_{m,n} / (2n - 1),
// whose Fourier symbol is i [k]_s (Eq. staggered_modified_wave_number); m = 1 is Yee's scheme.
// curl E is taken at the B positions (E is nodal along the axes it is differentiated along),
// curl B at the E positions.  One thread per cell; all three components of the updated field
// in one pass (HBM bound: the neighbours along x and y come from L2).
#include "pic_internal.cuh"

#include <cmath>

namespace {

template <class T>
struct FdW {
  int m;
  T c[PIC_MAX_CENTER_M];  // c_n / dx
};

template <class T>
struct FdtdArgs {
  T* F[3];         // field updated in place (B in the B pass, E in the E pass)
  const T* G[3];   // field differentiated (E in the B pass, B in the E pass)
  const T* J[3];   // E pass only
  int sh[3];       // log2 N per axis
  FdW<T> w[3];
  T h;             // time step of the pass: dt / 2 (B) or dt (E)
  T c2, eps0;
};

// Derivative along the axis of stride 2^s (coordinate j, N = mask + 1) of f around element e:
// HALF: f on the nodes of the axis, result at j + 1/2; else f on the half points (element i at
// i + 1/2), result at the node j.
template <class T, bool HALF>
__device__ __forceinline__ T dfd(const T* __restrict__ f, int e, int j, int mask, int s, const FdW<T>& w) {
  const int base = e - (j << s);
  T acc = T(0);
#pragma unroll
  for (int n = 1; n <= PIC_MAX_CENTER_M; ++n) {
    if (n > w.m) break;
    const int jp = (HALF ? j + n : j + n - 1) & mask;
    const int jm = (HALF ? j - n + 1 : j - n) & mask;
    acc += w.c[n - 1] * (f[base + (jp << s)] - f[base + (jm << s)]);
  }
  return acc;
}

// B pass: B -= h curl E (E: G, B: F).
template <class T>
__global__ void __launch_bounds__(256) fdtd_b_kernel(FdtdArgs<T> a) {
  const int ncell = 1 << (a.sh[0] + a.sh[1] + a.sh[2]);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const int sz = 0, sy = a.sh[2], sx = a.sh[1] + a.sh[2];
  const int mx = (1 << a.sh[0]) - 1, my = (1 << a.sh[1]) - 1, mz = (1 << a.sh[2]) - 1;
  const int iz = e & mz, iy = (e >> sy) & my, ix = e >> sx;
  const T* Ex = a.G[0];
  const T* Ey = a.G[1];
  const T* Ez = a.G[2];
  const T cx = dfd<T, true>(Ez, e, iy, my, sy, a.w[1]) - dfd<T, true>(Ey, e, iz, mz, sz, a.w[2]);
  const T cy = dfd<T, true>(Ex, e, iz, mz, sz, a.w[2]) - dfd<T, true>(Ez, e, ix, mx, sx, a.w[0]);
  const T cz = dfd<T, true>(Ey, e, ix, mx, sx, a.w[0]) - dfd<T, true>(Ex, e, iy, my, sy, a.w[1]);
  a.F[0][e] = a.F[0][e] - a.h * cx;
  a.F[1][e] = a.F[1][e] - a.h * cy;
  a.F[2][e] = a.F[2][e] - a.h * cz;
}

// E pass: E += h (c^2 curl B - J / eps0) (B: G, E: F).
template <class T>
__global__ void __launch_bounds__(256) fdtd_e_kernel(FdtdArgs<T> a) {
  const int ncell = 1 << (a.sh[0] + a.sh[1] + a.sh[2]);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  const int sz = 0, sy = a.sh[2], sx = a.sh[1] + a.sh[2];
  const int mx = (1 << a.sh[0]) - 1, my = (1 << a.sh[1]) - 1, mz = (1 << a.sh[2]) - 1;
  const int iz = e & mz, iy = (e >> sy) & my, ix = e >> sx;
  const T* Bx = a.G[0];
  const T* By = a.G[1];
  const T* Bz = a.G[2];
  const T cx = dfd<T, false>(Bz, e, iy, my, sy, a.w[1]) - dfd<T, false>(By, e, iz, mz, sz, a.w[2]);
  const T cy = dfd<T, false>(Bx, e, iz, mz, sz, a.w[2]) - dfd<T, false>(Bz, e, ix, mx, sx, a.w[0]);
  const T cz = dfd<T, false>(By, e, ix, mx, sx, a.w[0]) - dfd<T, false>(Bx, e, iy, my, sy, a.w[1]);
  a.F[0][e] = a.F[0][e] + a.h * (a.c2 * cx - a.J[0][e] / a.eps0);
  a.F[1][e] = a.F[1][e] + a.h * (a.c2 * cy - a.J[1][e] / a.eps0);
  a.F[2][e] = a.F[2][e] + a.h * (a.c2 * cz - a.J[2][e] / a.eps0);
}

int lg2(int64_t n) {
  int s = 0;
  while ((int64_t(1) << s) < n) ++s;
  return s;
}

template <class T>
FdtdArgs<T> make_args(const pic_ctx* ctx) {
  FdtdArgs<T> a;
  memset(&a, 0, sizeof(a));
  for (int d = 0; d < 3; ++d) {
    a.sh[d] = lg2(ctx->N[d]);
    a.w[d].m = ctx->fdw[d].m;
    for (int n = 0; n < ctx->fdw[d].m; ++n) a.w[d].c[n] = (T)ctx->fdw[d].w[n];
  }
  a.c2 = (T)(ctx->c * ctx->c);
  a.eps0 = (T)ctx->eps0;
  return a;
}

template <class T>
pic_status fdtd_update_t(pic_ctx* ctx, T* const E[3], T* const B[3], const T* const J[3]) {
  FdtdArgs<T> a = make_args<T>(ctx);
  const unsigned grid = (unsigned)((ctx->ncell + 255) / 256);
  StageScope t(ctx, STAGE_UPDATE, 3);
  // B^{n+1/2}
  for (int c = 0; c < 3; ++c) {
    a.F[c] = B[c];
    a.G[c] = E[c];
  }
  a.h = (T)(0.5 * ctx->dt);
  fdtd_b_kernel<T><<<grid, 256, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  // E^{n+1}
  for (int c = 0; c < 3; ++c) {
    a.F[c] = E[c];
    a.G[c] = B[c];
    a.J[c] = J[c];
  }
  a.h = (T)ctx->dt;
  fdtd_e_kernel<T><<<grid, 256, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  // B^{n+1}
  for (int c = 0; c < 3; ++c) {
    a.F[c] = B[c];
    a.G[c] = E[c];
    a.J[c] = nullptr;
  }
  a.h = (T)(0.5 * ctx->dt);
  fdtd_b_kernel<T><<<grid, 256, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

}  // namespace

pic_status fdtd_update(pic_ctx* ctx, double* const E[3], double* const B[3], const double* const J[3]) {
  return fdtd_update_t<double>(ctx, E, B, J);
}

pic_status fdtd_update32(pic_ctx* ctx, float* const E[3], float* const B[3], const float* const J[3]) {
  return fdtd_update_t<float>(ctx, E, B, J);
}

// FDTD weights c_n / dx per axis and the Courant check (host, at context creation).
pic_status fdtd_setup(pic_ctx* ctx) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int m = (ctx->sorder[a] ? ctx->sorder[a] : 2) / 2;
    ctx->fdw[a].m = m;
    long double ny = 0.0L;  // [k]_s at the Nyquist wave number: (2 / dx) sum_n c_n (-1)^(n+1)
    for (int n = 1; n <= m; ++n) {
      const long double cn = fornberg_alpha_s(m, n) / (2.0L * n - 1.0L) / (long double)ctx->dx[a];
      ctx->fdw[a].w[n - 1] = (double)cn;
      ny += (n % 2 ? 2.0L : -2.0L) * cn;
    }
    s += (double)(ny * ny);
  }
  if (ctx->c * ctx->dt * std::sqrt(s) > 2.0 * (1.0 + 1e-12))
    return pic_set_error(ctx, PIC_ERR_ARG, "dt %.6g is above the Courant limit %.6g of the FDTD solver", ctx->dt,
                         2.0 / (ctx->c * std::sqrt(s)));
  return PIC_OK;
}

// One call of the hybrid FDTD cycle, FP64: E, B (Yee) are the state and are advanced in place.
pic_status fdtd_step(pic_ctx* ctx, double* const E[3], double* const B[3], double* const J[3], double* rho,
                     const pic_species* sp, int n_species, int nsteps) {
  const int64_t nc = ctx->ncell;
  const double* En[3] = {ctx->nodal, ctx->nodal + nc, ctx->nodal + 2 * nc};
  const double* Bn[3] = {ctx->nodal + 3 * nc, ctx->nodal + 4 * nc, ctx->nodal + 5 * nc};
  double* Jn[3] = {ctx->Jn, ctx->Jn + nc, ctx->Jn + 2 * nc};
  double* nodal[6];
  for (int c = 0; c < 6; ++c) nodal[c] = ctx->nodal + c * nc;
  const double* yee[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  const double* cJn[3] = {Jn[0], Jn[1], Jn[2]};
  const double* cJ[3] = {J[0], J[1], J[2]};
  for (int s = 0; s < nsteps; ++s) {
    {
      // E^n, B^n -> nodes (scratch: ctx->Jn, free until the deposit)
      StageScope t(ctx, STAGE_OTHER, 9);
      PIC_TRY(center_to_nodal(ctx, yee, nodal));
    }
    if (ctx->sort_interval > 0 && ctx->steps_done % ctx->sort_interval == 0)
      for (int q = 0; q < n_species; ++q) {
        StageScope t(ctx, STAGE_BIN, sp[q].n > 0 ? 3 : 1);
        PIC_TRY(particles_bin(ctx, &sp[q], nullptr));
      }
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->Jn, 0, 3 * nc * sizeof(double), ctx->stream));
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho, 0, nc * sizeof(double), ctx->stream));
    for (int q = 0; q < n_species; ++q) {
      StageScope t(ctx, STAGE_PUSH, sp[q].n > 0 ? 1 : 0);
      PIC_TRY(particles_push(ctx, En, Bn, &sp[q], Jn, rho));
    }
    {
      // J^{n+1/2}: optional smoothing (Sec. 2), nodes -> Yee (work arrays: ctx->nodal, free after
      // the push)
      StageScope t(ctx, STAGE_OTHER, 3 + 9 * ctx->filter_passes);
      for (int c = 0; c < 3 && ctx->filter_passes > 0; ++c)
        PIC_TRY(bilinear_filter_t<double>(ctx, Jn[c], ctx->filter_passes, ctx->nodal, ctx->nodal + nc));
      PIC_TRY(center_to_yee(ctx, cJn, J));
    }
    PIC_TRY(fdtd_update(ctx, E, B, cJ));
    ++ctx->steps_done;
  }
  return PIC_OK;
}
