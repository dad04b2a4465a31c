// Reverse mode of the FP64 hybrid PIC step (pic_adjoint_step).
//
// The step is a composition of maps; its adjoint applies the transpose of each
// in reverse order: the PSATD update (per-mode conjugate transpose of the
// coefficient matrix, psatd.cu), the J centering (transpose = multiplication by
// zeta on the nodal spectrum), the deposits (transpose = gather of the adjoint
// densities, plus the B-spline derivative for positions), the move and v = u /
// gamma, the Boris push (reverse chain rule through its intermediates), the
// gather (transpose = deposit of the force adjoints, plus the shape derivative)
// and the E, B centering (transpose = zeta on the adjoint spectra).  Every
// forward quantity a transpose needs is recomputed from the state at t^n.
#include "pic_internal.cuh"

namespace {

struct AdjArgs {
  const double *x, *y, *z, *ux, *uy, *uz, *w;
  double *xb, *yb, *zb, *uxb, *uyb, *uzb;  // in: adjoints of x^{n+1}, u^{n+1/2}; out: of x^n, u^{n-1/2}
  int64_t n;
  const double* F[6];    // nodal E, B at t^n
  const double* Jb[3];   // nodal adjoint of J^{n+1/2}
  const double* Rb[2];   // nodal adjoints of rho^{n+1} (from the update and from the caller), summed
  double* Fb[6];         // nodal adjoints of the gathered E, B (atomic add)
  double inv_dx[3];
  double L[3];
  int mask[3];
  int64_t Ny, Nz;
  double k;              // q dt / (2 m)
  double dt;
  double inv_c2;
  double vg[3];
  double qw_scale;       // q / dV
};

// B-spline weights and their derivative in x (physical units), same cell rule as the forward.
template <int P>
__device__ __forceinline__ void shape_d(double x, double inv, int& lo, double* S, double* D) {
  const double t = __dmul_rn(x, inv);
  const double base = (P == 2) ? floor(__dadd_rn(t, 0.5)) : floor(t);
  const double d = t - base;
  const int b = (int)base;
  if (P == 1) {
    lo = b;
    S[0] = 1.0 - d;
    S[1] = d;
    D[0] = -inv;
    D[1] = inv;
  } else if (P == 2) {
    lo = b - 1;
    const double a = 0.5 - d, c = 0.5 + d;
    S[0] = 0.5 * a * a;
    S[1] = 0.75 - d * d;
    S[2] = 0.5 * c * c;
    D[0] = -a * inv;
    D[1] = -2.0 * d * inv;
    D[2] = c * inv;
  } else {
    lo = b - 1;
    const double e = 1.0 - d, d2 = d * d, d3 = d2 * d;
    S[0] = e * e * e * (1.0 / 6.0);
    S[1] = (4.0 - 6.0 * d2 + 3.0 * d3) * (1.0 / 6.0);
    S[2] = (1.0 + 3.0 * d + 3.0 * d2 - 3.0 * d3) * (1.0 / 6.0);
    S[3] = d3 * (1.0 / 6.0);
    D[0] = -0.5 * e * e * inv;
    D[1] = (-12.0 * d + 9.0 * d2) * (1.0 / 6.0) * inv;
    D[2] = (3.0 + 6.0 * d - 9.0 * d2) * (1.0 / 6.0) * inv;
    D[3] = 0.5 * d2 * inv;
  }
}

__device__ __forceinline__ double wrapd(double x, double L) {
  if (x >= L) x -= L;
  if (x < 0.0) x += L;
  return x;
}

// values and gradients of NF nodal arrays at a position
template <int P, int NF>
__device__ __forceinline__ void gather_grad(const AdjArgs& a, const double* const* F, double px, double py, double pz,
                                            double* val, double (*grad)[3]) {
  constexpr int NS = P + 1;
  int lx, ly, lz;
  double Sx[NS], Sy[NS], Sz[NS], Dx[NS], Dy[NS], Dz[NS];
  shape_d<P>(px, a.inv_dx[0], lx, Sx, Dx);
  shape_d<P>(py, a.inv_dx[1], ly, Sy, Dy);
  shape_d<P>(pz, a.inv_dx[2], lz, Sz, Dz);
#pragma unroll
  for (int c = 0; c < NF; ++c) {
    if (val) val[c] = 0.0;
    grad[c][0] = grad[c][1] = grad[c][2] = 0.0;
  }
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int64_t o = oy + ((lz + k) & a.mask[2]);
        const double s = Sx[i] * Sy[j] * Sz[k];
        const double g0 = Dx[i] * Sy[j] * Sz[k], g1 = Sx[i] * Dy[j] * Sz[k], g2 = Sx[i] * Sy[j] * Dz[k];
#pragma unroll
        for (int c = 0; c < NF; ++c) {
          const double f = __ldg(F[c] + o);
          if (val) val[c] += s * f;
          grad[c][0] += g0 * f;
          grad[c][1] += g1 * f;
          grad[c][2] += g2 * f;
        }
      }
    }
  }
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

template <int P>
__global__ void __launch_bounds__(128) adjoint_push_kernel(AdjArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const double x = a.x[p], y = a.y[p], z = a.z[p];
  const double u[3] = {a.ux[p], a.uy[p], a.uz[p]};
  const double qw = a.w[p] * a.qw_scale;
  // forward recompute: gather (with gradients) and Boris
  double F[6], dF[6][3];
  gather_grad<P, 6>(a, a.F, x, y, z, F, dF);
  const double k = a.k;
  double um[3], t[3], s[3], up[3], un[3];
  for (int c = 0; c < 3; ++c) um[c] = u[c] + k * F[c];
  const double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) * a.inv_c2);
  for (int c = 0; c < 3; ++c) t[c] = k * F[3 + c] / gm;
  const double ts = 1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int c = 0; c < 3; ++c) s[c] = 2.0 * t[c] / ts;
  double tmp[3];
  cross3(um, t, tmp);
  for (int c = 0; c < 3; ++c) up[c] = um[c] + tmp[c];
  cross3(up, s, tmp);
  for (int c = 0; c < 3; ++c) un[c] = um[c] + tmp[c] + k * F[c];
  const double g = sqrt(1.0 + (un[0] * un[0] + un[1] * un[1] + un[2] * un[2]) * a.inv_c2);
  double v[3];
  for (int c = 0; c < 3; ++c) v[c] = un[c] / g;
  const double mx = wrapd(x + 0.5 * a.dt * (v[0] - a.vg[0]), a.L[0]);
  const double my = wrapd(y + 0.5 * a.dt * (v[1] - a.vg[1]), a.L[1]);
  const double mz = wrapd(z + 0.5 * a.dt * (v[2] - a.vg[2]), a.L[2]);
  const double nx = wrapd(x + a.dt * (v[0] - a.vg[0]), a.L[0]);
  const double ny = wrapd(y + a.dt * (v[1] - a.vg[1]), a.L[1]);
  const double nz = wrapd(z + a.dt * (v[2] - a.vg[2]), a.L[2]);
  // deposits, reversed: gather the adjoint densities (and gradients) at x^{n+1/2}, x^{n+1}
  double Jv[3], dJ[3][3], dR[2][3];
  gather_grad<P, 3>(a, a.Jb, mx, my, mz, Jv, dJ);
  gather_grad<P, 2>(a, a.Rb, nx, ny, nz, nullptr, dR);
  double xnb[3], xmb[3], vb[3], xb[3];
  const double xin[3] = {a.xb[p], a.yb[p], a.zb[p]};
  for (int c = 0; c < 3; ++c) {
    xnb[c] = xin[c] + qw * (dR[0][c] + dR[1][c]);
    xmb[c] = qw * (v[0] * dJ[0][c] + v[1] * dJ[1][c] + v[2] * dJ[2][c]);
    vb[c] = qw * Jv[c] + 0.5 * a.dt * xmb[c] + a.dt * xnb[c];
    xb[c] = xnb[c] + xmb[c];
  }
  // v = u / gamma
  const double udv = (un[0] * vb[0] + un[1] * vb[1] + un[2] * vb[2]) * a.inv_c2 / (g * g * g);
  const double unb[3] = {a.uxb[p] + vb[0] / g - un[0] * udv, a.uyb[p] + vb[1] / g - un[1] * udv,
                         a.uzb[p] + vb[2] / g - un[2] * udv};
  // Boris, reversed
  double Eb[3], Bb[3], umb[3], upb[3], sb[3], tb[3];
  for (int c = 0; c < 3; ++c) Eb[c] = k * unb[c];
  cross3(s, unb, upb);        // upl = um + up x s
  cross3(unb, up, sb);
  for (int c = 0; c < 3; ++c) umb[c] = unb[c];
  cross3(t, upb, tmp);        // up = um + um x t
  for (int c = 0; c < 3; ++c) umb[c] += upb[c] + tmp[c];
  cross3(upb, um, tb);
  const double sdt = sb[0] * t[0] + sb[1] * t[1] + sb[2] * t[2];
  for (int c = 0; c < 3; ++c) tb[c] += 2.0 * sb[c] / ts - 4.0 * sdt / (ts * ts) * t[c];
  for (int c = 0; c < 3; ++c) Bb[c] = k / gm * tb[c];
  const double gmb = -(t[0] * tb[0] + t[1] * tb[1] + t[2] * tb[2]) / gm;
  for (int c = 0; c < 3; ++c) umb[c] += gmb * um[c] * a.inv_c2 / gm;
  for (int c = 0; c < 3; ++c) Eb[c] += k * umb[c];
  // gather, reversed: deposit the force adjoints at x^n; shape derivative for the position
  for (int c = 0; c < 3; ++c)
    xb[c] += Eb[0] * dF[0][c] + Eb[1] * dF[1][c] + Eb[2] * dF[2][c] + Bb[0] * dF[3][c] + Bb[1] * dF[4][c] +
             Bb[2] * dF[5][c];
  {
    constexpr int NS = P + 1;
    int lx, ly, lz;
    double Sx[NS], Sy[NS], Sz[NS], D[NS];
    shape_d<P>(x, a.inv_dx[0], lx, Sx, D);
    shape_d<P>(y, a.inv_dx[1], ly, Sy, D);
    shape_d<P>(z, a.inv_dx[2], lz, Sz, D);
    const double fb[6] = {Eb[0], Eb[1], Eb[2], Bb[0], Bb[1], Bb[2]};
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
#pragma unroll
        for (int kk = 0; kk < NS; ++kk) {
          const int64_t o = oy + ((lz + kk) & a.mask[2]);
          const double sw = Sx[i] * Sy[j] * Sz[kk];
#pragma unroll
          for (int c = 0; c < 6; ++c) atomicAdd(a.Fb[c] + o, sw * fb[c]);
        }
      }
    }
  }
  a.xb[p] = xb[0];
  a.yb[p] = xb[1];
  a.zb[p] = xb[2];
  a.uxb[p] = umb[0];
  a.uyb[p] = umb[1];
  a.uzb[p] = umb[2];
}

template <class P>
bool nonnull(P const* a, int n) {
  if (!a) return false;
  for (int i = 0; i < n; ++i)
    if (!a[i]) return false;
  return true;
}

#define ADJ_TRY(x)                 \
  do {                             \
    pic_status s_ = (x);           \
    if (s_ != PIC_OK) return s_;   \
  } while (0)

const int kKindEB[6] = {0, 1, 2, 3, 4, 5};

// Yee real arrays -> paper-convention spectra in ctx->EBh (through G)
pic_status to_paper(pic_ctx* ctx, const double* const* F6) {
  CRPtr6 in;
  CPtr6 g, eb;
  for (int c = 0; c < 6; ++c) {
    in.p[c] = F6[c];
    g.p[c] = ctx->G + c * ctx->nmode;
    eb.p[c] = ctx->EBh + c * ctx->nmode;
  }
  {
    StageScope t(ctx, STAGE_FFT, 3);
    ADJ_TRY(fft_r2c<double>(ctx, in, g, 6));
  }
  StageScope t(ctx, STAGE_OTHER, 1);
  return psatd_phase(ctx, g, eb, kKindEB, 6, -1, 1.0);
}

}  // namespace

extern "C" pic_status pic_adjoint_step(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                                       const pic_species* sp, int n_species, double* const Ebar[3],
                                       double* const Bbar[3], double* rhobar, const pic_species_adjoint* spbar) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "the adjoint step is FP64 only");
  if (ctx->variant == PIC_PSATD_AVERAGED_GALILEAN)
    return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "no adjoint for the averaged Galilean variant");
  if (ctx->filter_passes > 0 || ctx->pusher != PIC_PUSHER_BORIS || ctx->cycle != PIC_CYCLE_HYBRID)
    return pic_set_error(ctx, PIC_ERR_UNSUPPORTED,
                         "the adjoint covers the hybrid cycle with the Boris pusher and no smoothing");
  if (!nonnull(E, 3) || !nonnull(B, 3) || !nonnull(Ebar, 3) || !nonnull(Bbar, 3) || !rhobar)
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  {
    const void* ptrs[13] = {E[0], E[1], E[2], B[0], B[1], B[2], Ebar[0], Ebar[1], Ebar[2], Bbar[0], Bbar[1], Bbar[2],
                            rhobar};
    PIC_NEED_ALIGNED(ctx, ptrs, 13, 16);
  }
  if (n_species < 0 || (n_species > 0 && (!sp || !spbar))) return pic_set_error(ctx, PIC_ERR_ARG, "species");
  for (int s = 0; s < n_species; ++s) {
    if (sp[s].n != spbar[s].n) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: adjoint size mismatch", s);
    if (sp[s].n > 0 && (!sp[s].x || !sp[s].y || !sp[s].z || !sp[s].ux || !sp[s].uy || !sp[s].uz || !sp[s].w ||
                        !spbar[s].x || !spbar[s].y || !spbar[s].z || !spbar[s].ux || !spbar[s].uy || !spbar[s].uz))
      return pic_set_error(ctx, PIC_ERR_ARG, "species %d: null array", s);
    if (!(sp[s].m > 0.0)) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: mass must be > 0", s);
  }
  const int64_t nc = ctx->ncell, nm = ctx->nmode;
  if (!ctx->adj_work) {
    cudaError_t e = cudaMalloc(&ctx->adj_work, 8 * nc * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->adj_work = nullptr;
      return pic_set_error(ctx, PIC_ERR_NOMEM, "adjoint work arrays");
    }
  }
  double* rbn = ctx->adj_work;            // rhobar^n
  double* rbp = ctx->adj_work + nc;       // rhobar^{n+1} from the update
  double* fb = ctx->adj_work + 2 * nc;    // [6] nodal force adjoints
  // 1. nodal E, B at t^n (forward recompute)
  const double* F6[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  ADJ_TRY(to_paper(ctx, F6));
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    ADJ_TRY(psatd_to_nodal(ctx, ctx->EBh, 1.0 / (double)nc));
  }
  {
    CPtr6 g;
    RPtr6 o;
    for (int c = 0; c < 6; ++c) {
      g.p[c] = ctx->G + c * nm;
      o.p[c] = ctx->nodal + c * nc;
    }
    StageScope t(ctx, STAGE_FFT, 3);
    ADJ_TRY(fft_c2r<double>(ctx, g, o, 6));
  }
  // 2. transpose of the update on the incoming field adjoints
  const double* Fb6[6] = {Ebar[0], Ebar[1], Ebar[2], Bbar[0], Bbar[1], Bbar[2]};
  ADJ_TRY(to_paper(ctx, Fb6));
  {
    StageScope t(ctx, STAGE_UPDATE, 1);
    ADJ_TRY(psatd_adjoint_update(ctx, ctx->EBh, ctx->G));
  }
  {
    CPtr6 g;
    RPtr6 o;
    for (int c = 0; c < 5; ++c) g.p[c] = ctx->G + c * nm;
    for (int c = 0; c < 3; ++c) o.p[c] = ctx->Jn + c * nc;   // nodal Jbar
    o.p[3] = rbn;
    o.p[4] = rbp;
    StageScope t(ctx, STAGE_FFT, 3);
    ADJ_TRY(fft_c2r<double>(ctx, g, o, 5));
  }
  // 3. particles, reversed
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(fb, 0, 6 * nc * sizeof(double), ctx->stream));
  for (int s = 0; s < n_species; ++s) {
    if (sp[s].n == 0) continue;
    AdjArgs a;
    a.x = sp[s].x;
    a.y = sp[s].y;
    a.z = sp[s].z;
    a.ux = sp[s].ux;
    a.uy = sp[s].uy;
    a.uz = sp[s].uz;
    a.w = sp[s].w;
    a.xb = spbar[s].x;
    a.yb = spbar[s].y;
    a.zb = spbar[s].z;
    a.uxb = spbar[s].ux;
    a.uyb = spbar[s].uy;
    a.uzb = spbar[s].uz;
    a.n = sp[s].n;
    for (int c = 0; c < 6; ++c) {
      a.F[c] = ctx->nodal + c * nc;
      a.Fb[c] = fb + c * nc;
    }
    for (int c = 0; c < 3; ++c) a.Jb[c] = ctx->Jn + c * nc;
    a.Rb[0] = rbp;
    a.Rb[1] = rhobar;
    for (int d = 0; d < 3; ++d) {
      a.inv_dx[d] = 1.0 / ctx->dx[d];
      a.L[d] = (double)ctx->N[d] * ctx->dx[d];
      a.mask[d] = (int)ctx->N[d] - 1;
      a.vg[d] = ctx->variant == PIC_PSATD_STANDARD ? 0.0 : ctx->vg[d];
    }
    a.Ny = ctx->N[1];
    a.Nz = ctx->N[2];
    a.k = sp[s].q * ctx->dt / (2.0 * sp[s].m);
    a.dt = ctx->dt;
    a.inv_c2 = 1.0 / (ctx->c * ctx->c);
    a.qw_scale = sp[s].q / (ctx->dx[0] * ctx->dx[1] * ctx->dx[2]);
    const int bs = 128;
    const unsigned nb = (unsigned)((a.n + bs - 1) / bs);
    StageScope t(ctx, STAGE_PUSH, 1);
    switch (ctx->shape_order) {
      case 1: adjoint_push_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
      case 2: adjoint_push_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
      default: adjoint_push_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
    }
    PIC_LAUNCH_CHECK(ctx);
  }
  // 4. transpose of the E, B centering: EBh += zeta * DFT(force adjoints); back to Yee
  {
    CRPtr6 in;
    CPtr6 g;
    for (int c = 0; c < 6; ++c) {
      in.p[c] = fb + c * nc;
      g.p[c] = ctx->G + c * nm;
    }
    StageScope t(ctx, STAGE_FFT, 3);
    ADJ_TRY(fft_r2c<double>(ctx, in, g, 6));
  }
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    ADJ_TRY(psatd_add_zeta(ctx, ctx->EBh, ctx->G));
  }
  {
    CPtr6 s6, g;
    RPtr6 o;
    for (int c = 0; c < 6; ++c) {
      s6.p[c] = ctx->EBh + c * nm;
      g.p[c] = ctx->G + c * nm;
    }
    for (int c = 0; c < 3; ++c) {
      o.p[c] = Ebar[c];
      o.p[3 + c] = Bbar[c];
    }
    {
      StageScope t(ctx, STAGE_OTHER, 1);
      ADJ_TRY(psatd_phase(ctx, s6, g, kKindEB, 6, +1, 1.0 / (double)nc));
    }
    StageScope t(ctx, STAGE_FFT, 3);
    ADJ_TRY(fft_c2r<double>(ctx, g, o, 6));
  }
  // 5. adjoint of rho^n
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(rhobar, rbn, nc * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return PIC_OK;
}
