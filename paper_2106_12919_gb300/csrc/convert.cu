// Conversions between the FP64 and FP32 particle representations, and the adjoint seed of the
// probe-box field energy (the loss of the reverse mode).
//
// FP32-form positions: each coordinate is an integer cell i and an FP32 offset f in [0, 1) with
// x = (i + f) dx.  The split takes t = x * (1/dx) rounded to FP64 (the multiply of the FP64
// form's nearest-node rule), i = floor(t), f = t - i (exact in FP64) rounded once to FP32; an
// offset that rounds to 1.0 moves the particle to offset 0 of the next cell, and the cell wraps
// into [0, N).  The join is x = (i + f) * dx in FP64 (i + f is exact).  Products use __dmul_rn so
// that no multiply is contracted into an FMA: the results are the correctly rounded ones.
#include "pic_internal.cuh"

namespace {

struct SplitArgs {
  const double* x[3];
  const double* u[3];
  const double* w;
  const int64_t* id_in;
  int32_t* cell;
  float* f[3];
  float* u32[3];
  float* w32;
  int64_t* id_out;
  double inv_dx[3];
  int64_t N[3];
  int64_t n;
};

__global__ void split_kernel(SplitArgs a) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double t = __dmul_rn(a.x[d][p], a.inv_dx[d]);
      const double b = floor(t);
      float f = __double2float_rn(t - b);
      int64_t i = (int64_t)b;
      if (f == 1.0f) {
        f = 0.0f;
        i += 1;
      }
      i %= a.N[d];
      if (i < 0) i += a.N[d];
      idx[d] = i;
      a.f[d][p] = f;
      a.u32[d][p] = __double2float_rn(a.u[d][p]);
    }
    a.cell[p] = (int32_t)((idx[0] * a.N[1] + idx[1]) * a.N[2] + idx[2]);
    a.w32[p] = __double2float_rn(a.w[p]);
    if (a.id_out) a.id_out[p] = a.id_in[p];
  }
}

struct JoinArgs {
  const int32_t* cell;
  const float* f[3];
  const float* u32[3];
  const float* w32;
  const int64_t* id_in;
  double* x[3];
  double* u[3];
  double* w;
  int64_t* id_out;
  double dx[3];
  int64_t N[3];
  int64_t n;
};

__global__ void join_kernel(JoinArgs a) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = a.cell[p];
    const int64_t idx[3] = {c / (a.N[1] * a.N[2]), (c / a.N[2]) % a.N[1], c % a.N[2]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a.x[d][p] = __dmul_rn((double)idx[d] + (double)a.f[d][p], a.dx[d]);
      a.u[d][p] = (double)a.u32[d][p];
    }
    a.w[p] = (double)a.w32[p];
    if (a.id_out) a.id_out[p] = a.id_in[p];
  }
}

struct SeedArgs {
  const double* E[3];
  const double* B[3];
  double* Eb[3];
  double* Bb[3];
  int64_t lo[3], hi[3];
  int64_t N[3];
  int64_t ncell;
  double se, sb;
};

// Ebar = se E, Bbar = sb B on the cells of the box [lo, hi), 0 elsewhere.
__global__ void energy_seed_kernel(SeedArgs a) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < a.ncell;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t iz = m % a.N[2], r = m / a.N[2];
    const int64_t iy = r % a.N[1], ix = r / a.N[1];
    const bool in = ix >= a.lo[0] && ix < a.hi[0] && iy >= a.lo[1] && iy < a.hi[1] && iz >= a.lo[2] &&
                    iz < a.hi[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.Eb[c][m] = in ? a.se * a.E[c][m] : 0.0;
      a.Bb[c][m] = in ? a.sb * a.B[c][m] : 0.0;
    }
  }
}

int grid_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

pic_status species_pair_check(pic_ctx* ctx, const pic_species* s64, const pic_species32* s32) {
  if (!s64 || !s32) return pic_set_error(ctx, PIC_ERR_ARG, "null species");
  if (s64->n < 0 || s64->n != s32->n) return pic_set_error(ctx, PIC_ERR_ARG, "species counts differ or are negative");
  if (s64->n > ((int64_t)1 << 31) - 1) return pic_set_error(ctx, PIC_ERR_CAPACITY, "more than 2^31-1 particles");
  if (s64->n == 0) return PIC_OK;
  if (!s64->x || !s64->y || !s64->z || !s64->ux || !s64->uy || !s64->uz || !s64->w)
    return pic_set_error(ctx, PIC_ERR_ARG, "null FP64 species array");
  if (!s32->cell || !s32->fx || !s32->fy || !s32->fz || !s32->ux || !s32->uy || !s32->uz || !s32->w)
    return pic_set_error(ctx, PIC_ERR_ARG, "null FP32 species array");
  if ((s64->id == nullptr) != (s32->id == nullptr))
    return pic_set_error(ctx, PIC_ERR_ARG, "id given on one side only");
  return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_species32_from_species(pic_ctx* ctx, const pic_species* in, const pic_species32* out) {
  if (!ctx) return PIC_ERR_ARG;
  PIC_TRY(species_pair_check(ctx, in, out));
  if (in->n == 0) return PIC_OK;
  SplitArgs a;
  a.x[0] = in->x;
  a.x[1] = in->y;
  a.x[2] = in->z;
  a.u[0] = in->ux;
  a.u[1] = in->uy;
  a.u[2] = in->uz;
  a.w = in->w;
  a.id_in = in->id;
  a.cell = out->cell;
  a.f[0] = out->fx;
  a.f[1] = out->fy;
  a.f[2] = out->fz;
  a.u32[0] = out->ux;
  a.u32[1] = out->uy;
  a.u32[2] = out->uz;
  a.w32 = out->w;
  a.id_out = out->id;
  for (int d = 0; d < 3; ++d) {
    a.inv_dx[d] = 1.0 / ctx->dx[d];
    a.N[d] = ctx->N[d];
  }
  a.n = in->n;
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    split_kernel<<<grid_blocks(a.n), 256, 0, ctx->stream>>>(a);
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status pic_species32_to_species(pic_ctx* ctx, const pic_species32* in, const pic_species* out) {
  if (!ctx) return PIC_ERR_ARG;
  PIC_TRY(species_pair_check(ctx, out, in));
  if (in->n == 0) return PIC_OK;
  JoinArgs a;
  a.cell = in->cell;
  a.f[0] = in->fx;
  a.f[1] = in->fy;
  a.f[2] = in->fz;
  a.u32[0] = in->ux;
  a.u32[1] = in->uy;
  a.u32[2] = in->uz;
  a.w32 = in->w;
  a.id_in = in->id;
  a.x[0] = out->x;
  a.x[1] = out->y;
  a.x[2] = out->z;
  a.u[0] = out->ux;
  a.u[1] = out->uy;
  a.u[2] = out->uz;
  a.w = out->w;
  a.id_out = out->id;
  for (int d = 0; d < 3; ++d) {
    a.dx[d] = ctx->dx[d];
    a.N[d] = ctx->N[d];
  }
  a.n = in->n;
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    join_kernel<<<grid_blocks(a.n), 256, 0, ctx->stream>>>(a);
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status pic_field_energy_adjoint(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                                    const int64_t box_lo[3], const int64_t box_hi[3], double scale,
                                    double* const Ebar[3], double* const Bbar[3]) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "pic_field_energy_adjoint needs an FP64 context");
  if (!E || !B || !Ebar || !Bbar) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  for (int c = 0; c < 3; ++c)
    if (!E[c] || !B[c] || !Ebar[c] || !Bbar[c]) return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  if ((box_lo == nullptr) != (box_hi == nullptr)) return pic_set_error(ctx, PIC_ERR_ARG, "give both box corners or neither");
  SeedArgs a;
  for (int d = 0; d < 3; ++d) {
    a.lo[d] = 0;
    a.hi[d] = ctx->N[d];
    a.N[d] = ctx->N[d];
    if (box_lo) {
      if (box_lo[d] < 0 || box_hi[d] > ctx->N[d] || box_lo[d] > box_hi[d])
        return pic_set_error(ctx, PIC_ERR_ARG, "box out of range");
      a.lo[d] = box_lo[d];
      a.hi[d] = box_hi[d];
    }
  }
  for (int c = 0; c < 3; ++c) {
    a.E[c] = E[c];
    a.B[c] = B[c];
    a.Eb[c] = Ebar[c];
    a.Bb[c] = Bbar[c];
  }
  a.ncell = ctx->ncell;
  // W = 1/2 sum (eps0 |E|^2 + |B|^2 / mu0) dV with 1 / mu0 = eps0 c^2
  const double dV = ctx->dx[0] * ctx->dx[1] * ctx->dx[2];
  a.se = scale * ctx->eps0 * dV;
  a.sb = scale * ctx->eps0 * ctx->c * ctx->c * dV;
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    energy_seed_kernel<<<grid_blocks(a.ncell), 256, 0, ctx->stream>>>(a);
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

}  // extern "C"
