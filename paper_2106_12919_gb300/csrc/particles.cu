// Particle stage of the hybrid cycle (Sec. 2): gather E, B from the nodal grid
// with B-spline shapes, Boris push, move, direct deposition of J^{n+1/2} and
// rho^{n+1} on the nodal grid; and tile binning of the particle SoA.
//
// Shapes (textbook centred B-splines on the nodal grid, node i at i dx):
//   order 1: base = floor(t), d = t - base; nodes base..base+1
//   order 2: base = floor(t + 1/2);          nodes base-1..base+1
//   order 3: base = floor(t);                nodes base-1..base+2
// with t = x * (1/dx) as one correctly rounded multiply (__dmul_rn) so that the
// integer cell decision is the same on every implementation.
// Node indices wrap with & (N - 1) (N a power of two), which also keeps every
// access in bounds whatever the position value.
#include "pic_internal.cuh"

namespace {

struct PushArgs {
  double *x, *y, *z, *ux, *uy, *uz;
  const double* w;
  int64_t n;
  const double* F[6];  // nodal Ex, Ey, Ez, Bx, By, Bz
  double* J[3];        // nodal J deposit (atomic add)
  double* rho;         // nodal rho deposit (atomic add)
  double inv_dx[3];
  double L[3];
  int mask[3];
  int64_t Ny, Nz;
  double qm_half_dt;   // q dt / (2 m)
  double dt;
  double inv_c2;
  double vg[3];
  double qw_scale;     // q / dV
  int gather;          // 0: rho-only deposit at the current position
  int vay;             // 1: Vay's pusher instead of Boris
};

// shape of order P at position x on a grid whose points sit at (i + off) dx (off = 0: nodes,
// off = 1/2: a staggered Yee axis): t = x / dx - off
template <int P>
__device__ __forceinline__ void shape(double x, double inv, int mask, int& lo, double* S, double off = 0.0) {
  const double t = __dmul_rn(x, inv) - off;
  double base;
  if (P == 2) base = floor(__dadd_rn(t, 0.5));
  else base = floor(t);
  const double d = t - base;
  const int b = (int)base;
  if (P == 1) {
    lo = b;
    S[0] = 1.0 - d;
    S[1] = d;
  } else if (P == 2) {
    lo = b - 1;
    const double a = 0.5 - d, c = 0.5 + d;
    S[0] = 0.5 * a * a;
    S[1] = 0.75 - d * d;
    S[2] = 0.5 * c * c;
  } else {
    lo = b - 1;
    const double e = 1.0 - d, d2 = d * d, d3 = d2 * d;
    S[0] = e * e * e * (1.0 / 6.0);
    S[1] = (4.0 - 6.0 * d2 + 3.0 * d3) * (1.0 / 6.0);
    S[2] = (1.0 + 3.0 * d + 3.0 * d2 - 3.0 * d3) * (1.0 / 6.0);
    S[3] = d3 * (1.0 / 6.0);
  }
  (void)mask;
}

// u^{n-1/2} of particle p -> u^{n+1/2} with the gathered f = (E, B): Boris rotation, or Vay's pusher
__device__ __forceinline__ void push_u(const PushArgs& a, int64_t p, const double* f, double& ux, double& uy,
                                       double& uz) {
  const double k = a.qm_half_dt;
  if (a.vay) {
    ux = a.ux[p];
    uy = a.uy[p];
    uz = a.uz[p];
    vay_push<double>(ux, uy, uz, f, k, a.inv_c2);
    return;
  }
  const double umx = a.ux[p] + k * f[0], umy = a.uy[p] + k * f[1], umz = a.uz[p] + k * f[2];
  const double gm = sqrt(1.0 + (umx * umx + umy * umy + umz * umz) * a.inv_c2);
  const double tx = k * f[3] / gm, ty = k * f[4] / gm, tz = k * f[5] / gm;
  const double s2 = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
  const double sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
  const double upx = umx + (umy * tz - umz * ty);
  const double upy = umy + (umz * tx - umx * tz);
  const double upz = umz + (umx * ty - umy * tx);
  ux = umx + (upy * sz - upz * sy) + k * f[0];
  uy = umy + (upz * sx - upx * sz) + k * f[1];
  uz = umz + (upx * sy - upy * sx) + k * f[2];
}

__device__ __forceinline__ double wrap(double x, double L) {
  if (x >= L) x -= L;
  if (x < 0.0) x += L;
  return x;
}

// rho of one particle: node (i, j, k) receives (Sx_i q w)(Sy_j Sz_k); Syz is the caller's storage
template <int P>
__device__ __forceinline__ void deposit_rho_nodes(const PushArgs& a, int lx, int ly, int lz, const double* Sx,
                                                  const double* Sy, const double* Sz, double qw,
                                                  double (&Syz)[P + 1][P + 1]) {
  constexpr int NS = P + 1;
  double Sq[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) Sq[i] = Sx[i] * qw;
#pragma unroll
  for (int j = 0; j < NS; ++j)
#pragma unroll
    for (int k = 0; k < NS; ++k) Syz[j][k] = Sy[j] * Sz[k];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
#pragma unroll
      for (int k = 0; k < NS; ++k) atomicAdd(a.rho + oy + ((lz + k) & a.mask[2]), Sq[i] * Syz[j][k]);
    }
  }
}

template <int P>
__device__ __forceinline__ void push_particle(const PushArgs& a, int64_t p) {
  constexpr int NS = P + 1;
  const double x = a.x[p], y = a.y[p], z = a.z[p];
  const double qw = a.w[p] * a.qw_scale;
  int lx, ly, lz;
  double Sx[NS], Sy[NS], Sz[NS];
  // The weight of node (i, j, k) is Sx_i Sy_j Sz_k.  Every sum below forms the NS^2 products
  // Sy_j Sz_k once and carries the particle's factor (q w, or q w v_c) on the NS x weights, so a
  // node costs one FP64 multiply or FMA per value instead of two (the FP64 pipe bounds this kernel).
  double Syz[NS][NS];
  if (!a.gather) {
    shape<P>(x, a.inv_dx[0], a.mask[0], lx, Sx);
    shape<P>(y, a.inv_dx[1], a.mask[1], ly, Sy);
    shape<P>(z, a.inv_dx[2], a.mask[2], lz, Sz);
    deposit_rho_nodes<P>(a, lx, ly, lz, Sx, Sy, Sz, qw, Syz);
    return;
  }
  shape<P>(x, a.inv_dx[0], a.mask[0], lx, Sx);
  shape<P>(y, a.inv_dx[1], a.mask[1], ly, Sy);
  shape<P>(z, a.inv_dx[2], a.mask[2], lz, Sz);
  // gather E, B at x^n: f_c = sum_i Sx_i g_ic, g_ic = sum_jk (Sy_j Sz_k) F_c(i, j, k)
#pragma unroll
  for (int j = 0; j < NS; ++j)
#pragma unroll
    for (int k = 0; k < NS; ++k) Syz[j][k] = Sy[j] * Sz[k];
  double f[6];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
    double g[6];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int64_t o = oy + ((lz + k) & a.mask[2]);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const double v = __ldg(a.F[c] + o);
          g[c] = (j == 0 && k == 0) ? Syz[j][k] * v : fma(Syz[j][k], v, g[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) f[c] = i == 0 ? Sx[0] * g[c] : fma(Sx[i], g[c], f[c]);
  }
  // push u^{n-1/2} -> u^{n+1/2}
  double ux, uy, uz;
  push_u(a, p, f, ux, uy, uz);
  const double ig = 1.0 / sqrt(1.0 + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
  const double vx = ux * ig, vy = uy * ig, vz = uz * ig;
  // move: x^{n+1} = x^n + dt (v - v_gal); J at x^{n+1/2}
  const double dX = a.dt * (vx - a.vg[0]), dY = a.dt * (vy - a.vg[1]), dZ = a.dt * (vz - a.vg[2]);
  const double mx = wrap(x + 0.5 * dX, a.L[0]), my = wrap(y + 0.5 * dY, a.L[1]), mz = wrap(z + 0.5 * dZ, a.L[2]);
  const double nx = wrap(x + dX, a.L[0]), ny = wrap(y + dY, a.L[1]), nz = wrap(z + dZ, a.L[2]);
  a.x[p] = nx;
  a.y[p] = ny;
  a.z[p] = nz;
  a.ux[p] = ux;
  a.uy[p] = uy;
  a.uz[p] = uz;
  // J^{n+1/2} = q w v S(x^{n+1/2} - x_i) / dV
  shape<P>(mx, a.inv_dx[0], a.mask[0], lx, Sx);
  shape<P>(my, a.inv_dx[1], a.mask[1], ly, Sy);
  shape<P>(mz, a.inv_dx[2], a.mask[2], lz, Sz);
  const double jx = qw * vx, jy = qw * vy, jz = qw * vz;
  double Sj[3][NS];  // (Sx_i q w v_c)
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    Sj[0][i] = Sx[i] * jx;
    Sj[1][i] = Sx[i] * jy;
    Sj[2][i] = Sx[i] * jz;
  }
#pragma unroll
  for (int j = 0; j < NS; ++j)
#pragma unroll
    for (int k = 0; k < NS; ++k) Syz[j][k] = Sy[j] * Sz[k];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
#pragma unroll
      for (int kk = 0; kk < NS; ++kk) {
        const int64_t o = oy + ((lz + kk) & a.mask[2]);
        atomicAdd(a.J[0] + o, Sj[0][i] * Syz[j][kk]);
        atomicAdd(a.J[1] + o, Sj[1][i] * Syz[j][kk]);
        atomicAdd(a.J[2] + o, Sj[2][i] * Syz[j][kk]);
      }
    }
  }
  // rho^{n+1} = q w S(x^{n+1} - x_i) / dV
  shape<P>(nx, a.inv_dx[0], a.mask[0], lx, Sx);
  shape<P>(ny, a.inv_dx[1], a.mask[1], ly, Sy);
  shape<P>(nz, a.inv_dx[2], a.mask[2], lz, Sz);
  deposit_rho_nodes<P>(a, lx, ly, lz, Sx, Sy, Sz, qw, Syz);
}

// The cubic form holds 128 registers (2 CTAs of 256 threads per SM, no spills); orders 1 and 2 keep
// the compiler's own choice (64 and ~100 registers).
template <int P>
__global__ void __launch_bounds__(256) push_kernel(PushArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < a.n) push_particle<P>(a, p);
}
template <>
__global__ void __launch_bounds__(256, 2) push_kernel<3>(PushArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < a.n) push_particle<3>(a, p);
}

// Staggered comparison cycle (Sec. 2): E, B are gathered from their own Yee positions and J is
// deposited at its Yee positions (rho stays nodal).  Component c is staggered along the axes of
// its bit mask (E: x, y, z; B: yz, xz, xy); shapes on the staggered axes use offset 1/2.
template <int P>
__device__ __forceinline__ double gather_one(const double* F, const PushArgs& a, const int* lo, const double* Sx,
                                             const double* Sy, const double* Sz) {
  constexpr int NS = P + 1;
  double v = 0.0;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lo[0] + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((lo[1] + j) & a.mask[1])) * a.Nz;
      const double sxy = Sx[i] * Sy[j];
#pragma unroll
      for (int k = 0; k < NS; ++k) v += sxy * Sz[k] * __ldg(F + oy + ((lo[2] + k) & a.mask[2]));
    }
  }
  return v;
}

template <int P>
__device__ __forceinline__ void deposit_one(double* F, const PushArgs& a, const int* lo, const double* Sx,
                                            const double* Sy, const double* Sz, double val) {
  constexpr int NS = P + 1;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lo[0] + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((lo[1] + j) & a.mask[1])) * a.Nz;
      const double sxy = Sx[i] * Sy[j] * val;
#pragma unroll
      for (int k = 0; k < NS; ++k) atomicAdd(F + oy + ((lo[2] + k) & a.mask[2]), sxy * Sz[k]);
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) push_stag_kernel(PushArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  constexpr int NS = P + 1;
  const double x[3] = {a.x[p], a.y[p], a.z[p]};
  const double qw = a.w[p] * a.qw_scale;
  // shapes on the nodal (0) and staggered (1) grid of every axis
  int l0[3], l1[3];
  double S0[3][NS], S1[3][NS];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    shape<P>(x[d], a.inv_dx[d], a.mask[d], l0[d], S0[d], 0.0);
    shape<P>(x[d], a.inv_dx[d], a.mask[d], l1[d], S1[d], 0.5);
  }
  constexpr int kStag[6] = {1, 2, 4, 6, 5, 3};  // Ex, Ey, Ez, Bx, By, Bz
  double f[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int m = kStag[c];
    const int lo[3] = {(m & 1) ? l1[0] : l0[0], (m & 2) ? l1[1] : l0[1], (m & 4) ? l1[2] : l0[2]};
    f[c] = gather_one<P>(a.F[c], a, lo, (m & 1) ? S1[0] : S0[0], (m & 2) ? S1[1] : S0[1], (m & 4) ? S1[2] : S0[2]);
  }
  double ux, uy, uz;
  push_u(a, p, f, ux, uy, uz);
  const double ig = 1.0 / sqrt(1.0 + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
  const double v[3] = {ux * ig, uy * ig, uz * ig};
  double mid[3], nw[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double dd = a.dt * (v[d] - a.vg[d]);
    mid[d] = wrap(x[d] + 0.5 * dd, a.L[d]);
    nw[d] = wrap(x[d] + dd, a.L[d]);
  }
  a.x[p] = nw[0];
  a.y[p] = nw[1];
  a.z[p] = nw[2];
  a.ux[p] = ux;
  a.uy[p] = uy;
  a.uz[p] = uz;
  // J^{n+1/2}: component d at its Yee positions (staggered along axis d)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    shape<P>(mid[d], a.inv_dx[d], a.mask[d], l0[d], S0[d], 0.0);
    shape<P>(mid[d], a.inv_dx[d], a.mask[d], l1[d], S1[d], 0.5);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lo[3] = {c == 0 ? l1[0] : l0[0], c == 1 ? l1[1] : l0[1], c == 2 ? l1[2] : l0[2]};
    deposit_one<P>(a.J[c], a, lo, c == 0 ? S1[0] : S0[0], c == 1 ? S1[1] : S0[1], c == 2 ? S1[2] : S0[2],
                   qw * v[c]);
  }
  // rho^{n+1} on the nodes
#pragma unroll
  for (int d = 0; d < 3; ++d) shape<P>(nw[d], a.inv_dx[d], a.mask[d], l0[d], S0[d], 0.0);
  deposit_one<P>(a.rho, a, l0, S0[0], S0[1], S0[2], qw);
}

PushArgs make_args(pic_ctx* ctx, const pic_species* sp) {
  PushArgs a;
  a.x = sp->x;
  a.y = sp->y;
  a.z = sp->z;
  a.ux = sp->ux;
  a.uy = sp->uy;
  a.uz = sp->uz;
  a.w = sp->w;
  a.n = sp->n;
  for (int d = 0; d < 3; ++d) {
    a.inv_dx[d] = 1.0 / ctx->dx[d];
    a.L[d] = (double)ctx->N[d] * ctx->dx[d];
    a.mask[d] = (int)ctx->N[d] - 1;
    a.vg[d] = ctx->variant == PIC_PSATD_STANDARD ? 0.0 : ctx->vg[d];
  }
  a.Ny = ctx->N[1];
  a.Nz = ctx->N[2];
  a.qm_half_dt = sp->q * ctx->dt / (2.0 * sp->m);
  a.dt = ctx->dt;
  a.inv_c2 = 1.0 / (ctx->c * ctx->c);
  a.vay = ctx->pusher == PIC_PUSHER_VAY ? 1 : 0;
  a.qw_scale = sp->q / (ctx->dx[0] * ctx->dx[1] * ctx->dx[2]);
  return a;
}

pic_status launch_push(pic_ctx* ctx, const PushArgs& a) {
  if (a.n == 0) return PIC_OK;
  const int bs = 256;
  const unsigned nb = (unsigned)((a.n + bs - 1) / bs);
  if (a.gather && ctx->cycle == PIC_CYCLE_STAGGERED) {
    switch (ctx->shape_order) {
      case 1: push_stag_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
      case 2: push_stag_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
      default: push_stag_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
    }
    PIC_LAUNCH_CHECK(ctx);
    return PIC_OK;
  }
  switch (ctx->shape_order) {
    case 1: push_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
    case 2: push_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
    default: push_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// tile binning
// ---------------------------------------------------------------------------
struct BinArgs {
  const double *x, *y, *z;
  int64_t n;
  double inv_dx[3];
  int mask[3];
  int tshift[3];  // log2 of the tile edge
  int64_t nty, ntz;
  int32_t* tid;
  unsigned long long* counts;
};

__global__ void tile_id_kernel(BinArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int cx = (int)floor(__dmul_rn(a.x[p], a.inv_dx[0])) & a.mask[0];
  const int cy = (int)floor(__dmul_rn(a.y[p], a.inv_dx[1])) & a.mask[1];
  const int cz = (int)floor(__dmul_rn(a.z[p], a.inv_dx[2])) & a.mask[2];
  const int t = (int)(((cx >> a.tshift[0]) * a.nty + (cy >> a.tshift[1])) * a.ntz + (cz >> a.tshift[2]));
  a.tid[p] = t;
  // warp-aggregated histogram
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, t);
  const int leader = __ffs(peers) - 1;
  if ((int)(threadIdx.x & 31) == leader) atomicAdd(a.counts + t, (unsigned long long)__popc(peers));
}

// Exclusive scan of n counts into off[0..n] by one CTA (n up to a few million).
__global__ void __launch_bounds__(1024) scan_kernel(const unsigned long long* cnt, int64_t* off, int64_t n) {
  __shared__ unsigned long long part[1024];
  const int T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t b = threadIdx.x * chunk, e = min(n, b + chunk);
  unsigned long long s = 0;
  for (int64_t i = b; i < e; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < T; d <<= 1) {
    unsigned long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0ull;
  for (int64_t i = b; i < e; ++i) {
    off[i] = (int64_t)run;
    run += cnt[i];
  }
  if (threadIdx.x == T - 1) off[n] = (int64_t)part[T - 1];
}

struct ScatterArgs {
  const double* src[8];  // x y z ux uy uz w id(as double bits)
  double* dst[8];
  int nfield;
  int64_t n;
  const int32_t* tid;
  const int64_t* off;
  unsigned long long* cursor;
};

__global__ void scatter_kernel(ScatterArgs a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int t = a.tid[p];
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, t);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(a.cursor + t, (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int64_t q = a.off[t] + (int64_t)base + rank;
  for (int f = 0; f < a.nfield; ++f) a.dst[f][q] = a.src[f][p];
}

pic_status ensure_bin_capacity(pic_ctx* ctx, int64_t n) {
  if (ctx->bin_counts == nullptr) {
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->bin_counts, (ctx->n_tiles + 1) * sizeof(int64_t)));
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->bin_cursor, ctx->n_tiles * sizeof(int64_t)));
  }
  if (n <= ctx->bin_cap) return PIC_OK;
  cudaFree(ctx->bin_tid);
  cudaFree(ctx->bin_tmp);
  ctx->bin_tid = nullptr;
  ctx->bin_tmp = nullptr;
  ctx->bin_cap = 0;
  if (cudaMalloc(&ctx->bin_tid, n * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&ctx->bin_tmp, 8 * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return pic_set_error(ctx, PIC_ERR_NOMEM, "binning scratch for %lld particles", (long long)n);
  }
  ctx->bin_cap = n;
  return PIC_OK;
}

int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

}  // namespace

pic_status particles_bin_capacity(pic_ctx* ctx, int64_t n) { return ensure_bin_capacity(ctx, n); }

pic_status particles_push(pic_ctx* ctx, const double* const En[3], const double* const Bn[3],
                          const pic_species* sp, double* const J[3], double* rho) {
  PushArgs a = make_args(ctx, sp);
  for (int c = 0; c < 3; ++c) {
    a.F[c] = En[c];
    a.F[3 + c] = Bn[c];
    a.J[c] = J[c];
  }
  a.rho = rho;
  a.gather = 1;
  return launch_push(ctx, a);
}

pic_status particles_deposit_rho(pic_ctx* ctx, const pic_species* sp, double* rho) {
  PushArgs a = make_args(ctx, sp);
  for (int c = 0; c < 6; ++c) a.F[c] = nullptr;
  for (int c = 0; c < 3; ++c) a.J[c] = nullptr;
  a.rho = rho;
  a.gather = 0;
  return launch_push(ctx, a);
}

pic_status particles_bin(pic_ctx* ctx, const pic_species* sp, int64_t* offsets_out) {
  const int64_t n = sp->n;
  pic_status st = ensure_bin_capacity(ctx, n > 0 ? n : 1);
  if (st != PIC_OK) return st;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctx->bin_cursor);
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, ctx->n_tiles * sizeof(int64_t), ctx->stream));
  BinArgs b;
  b.x = sp->x;
  b.y = sp->y;
  b.z = sp->z;
  b.n = n;
  for (int d = 0; d < 3; ++d) {
    b.inv_dx[d] = 1.0 / ctx->dx[d];
    b.mask[d] = (int)ctx->N[d] - 1;
    b.tshift[d] = ilog2(ctx->tile[d]);
  }
  b.nty = ctx->N[1] / ctx->tile[1];
  b.ntz = ctx->N[2] / ctx->tile[2];
  b.tid = ctx->bin_tid;
  b.counts = cnt;
  const int bs = 256;
  const unsigned nb = (unsigned)((n + bs - 1) / bs);
  if (n > 0) {
    tile_id_kernel<<<nb, bs, 0, ctx->stream>>>(b);
    PIC_LAUNCH_CHECK(ctx);
  }
  scan_kernel<<<1, 1024, 0, ctx->stream>>>(cnt, ctx->bin_counts, ctx->n_tiles);
  PIC_LAUNCH_CHECK(ctx);
  if (offsets_out)
    PIC_CUDA_TRY(ctx, cudaMemcpyAsync(offsets_out, ctx->bin_counts, (ctx->n_tiles + 1) * sizeof(int64_t),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
  if (n == 0) return PIC_OK;
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, ctx->n_tiles * sizeof(int64_t), ctx->stream));
  ScatterArgs s;
  double* fields[8] = {sp->x, sp->y, sp->z, sp->ux, sp->uy, sp->uz, sp->w, reinterpret_cast<double*>(sp->id)};
  s.nfield = sp->id ? 8 : 7;
  for (int f = 0; f < s.nfield; ++f) {
    s.src[f] = fields[f];
    s.dst[f] = ctx->bin_tmp + (int64_t)f * ctx->bin_cap;
  }
  s.n = n;
  s.tid = ctx->bin_tid;
  s.off = ctx->bin_counts;
  s.cursor = cnt;
  scatter_kernel<<<nb, bs, 0, ctx->stream>>>(s);
  PIC_LAUNCH_CHECK(ctx);
  for (int f = 0; f < s.nfield; ++f)
    PIC_CUDA_TRY(ctx, cudaMemcpyAsync(fields[f], s.dst[f], n * sizeof(double), cudaMemcpyDeviceToDevice,
                                      ctx->stream));
  return PIC_OK;
}
