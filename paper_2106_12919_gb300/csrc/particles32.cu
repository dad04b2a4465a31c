// Particle stage of the FP32 form: positions are an int32 linear cell index
// plus FP32 offsets in [0, 1) inside that cell; momenta, weights, nodal fields
// and deposits are FP32.  Same cycle as the FP64 form (Sec. 2): gather E, B at
// x^n from the nodal grid, Boris push, move by dt (v - v_gal), direct
// deposition of J^{n+1/2} at x^{n+1/2} and rho^{n+1} at x^{n+1}.
//
// Cell index c = (ix * Ny + iy) * Nz + iz; the cell decisions are integer
// (the offset crossing 0 or 1 moves the cell by one), so the FP32 form keeps
// sub-cell resolution of 2^-24 cells anywhere in the box.
#include "pic_internal.cuh"

namespace {

struct Push32Args {
  int32_t* cell;
  float *fx, *fy, *fz, *ux, *uy, *uz;
  const float* w;
  int64_t n;
  const float* F[6];  // nodal Ex, Ey, Ez, Bx, By, Bz
  float* J[3];
  float* rho;
  int shz, shy;       // log2 Nz, log2 Ny
  int mask[3];
  int64_t Ny, Nz;
  float qm_half_dt;   // q dt / (2 m)
  float inv_c2;
  float dtdx[3];      // dt / dx_a
  float vg[3];
  float qw_scale;     // q / dV
  int gather;
};

// shape of order P from the base cell i and the offset f in [0, 1)
template <int P>
__device__ __forceinline__ void shape32(int i, float f, int& lo, float* S) {
  if (P == 1) {
    lo = i;
    S[0] = 1.0f - f;
    S[1] = f;
  } else if (P == 2) {
    // nearest node: base = i (f < 1/2) or i + 1; d = f - (base - i) in [-1/2, 1/2)
    const bool up = f >= 0.5f;
    const float d = up ? f - 1.0f : f;
    lo = (up ? i + 1 : i) - 1;
    const float a = 0.5f - d, c = 0.5f + d;
    S[0] = 0.5f * a * a;
    S[1] = 0.75f - d * d;
    S[2] = 0.5f * c * c;
  } else {
    lo = i - 1;
    const float e = 1.0f - f, d2 = f * f, d3 = d2 * f;
    S[0] = e * e * e * (1.0f / 6.0f);
    S[1] = (4.0f - 6.0f * d2 + 3.0f * d3) * (1.0f / 6.0f);
    S[2] = (1.0f + 3.0f * f + 3.0f * d2 - 3.0f * d3) * (1.0f / 6.0f);
    S[3] = d3 * (1.0f / 6.0f);
  }
}

// offset f moved by d cells: new (cell shift, offset in [0, 1))
__device__ __forceinline__ int move_offset(float f, float d, float& out) {
  const float g = f + d;
  const float fl = floorf(g);
  float r = g - fl;
  int s = (int)fl;
  if (r >= 1.0f) {  // g just below an integer rounded up
    r = 0.0f;
    s += 1;
  }
  out = r;
  return s;
}

template <int P>
__device__ __forceinline__ void deposit_node_block(const Push32Args& a, int ix, int iy, int iz, float fx, float fy,
                                                   float fz, float v0, float v1, float v2, float r, bool j) {
  constexpr int NS = P + 1;
  int lx, ly, lz;
  float Sx[NS], Sy[NS], Sz[NS];
  shape32<P>(ix, fx, lx, Sx);
  shape32<P>(iy, fy, ly, Sy);
  shape32<P>(iz, fz, lz, Sz);
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int jj = 0; jj < NS; ++jj) {
      const int64_t oy = (ox + ((ly + jj) & a.mask[1])) * a.Nz;
      const float sxy = Sx[i] * Sy[jj];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int64_t o = oy + ((lz + k) & a.mask[2]);
        const float s = sxy * Sz[k];
        if (j) {
          atomicAdd(a.J[0] + o, s * v0);
          atomicAdd(a.J[1] + o, s * v1);
          atomicAdd(a.J[2] + o, s * v2);
        } else {
          atomicAdd(a.rho + o, s * r);
        }
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) push32_kernel(Push32Args a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  constexpr int NS = P + 1;
  const int c = a.cell[p];
  int ix = c >> (a.shz + a.shy), iy = (c >> a.shz) & a.mask[1], iz = c & a.mask[2];
  ix &= a.mask[0];
  const float fx = a.fx[p], fy = a.fy[p], fz = a.fz[p];
  const float qw = a.w[p] * a.qw_scale;
  if (!a.gather) {
    deposit_node_block<P>(a, ix, iy, iz, fx, fy, fz, 0.f, 0.f, 0.f, qw, false);
    return;
  }
  int lx, ly, lz;
  float Sx[NS], Sy[NS], Sz[NS];
  shape32<P>(ix, fx, lx, Sx);
  shape32<P>(iy, fy, ly, Sy);
  shape32<P>(iz, fz, lz, Sz);
  float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lx + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((ly + j) & a.mask[1])) * a.Nz;
      const float sxy = Sx[i] * Sy[j];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int64_t o = oy + ((lz + k) & a.mask[2]);
        const float s = sxy * Sz[k];
#pragma unroll
        for (int q = 0; q < 6; ++q) f[q] += s * __ldg(a.F[q] + o);
      }
    }
  }
  // Boris push u^{n-1/2} -> u^{n+1/2}
  const float kq = a.qm_half_dt;
  const float umx = a.ux[p] + kq * f[0], umy = a.uy[p] + kq * f[1], umz = a.uz[p] + kq * f[2];
  const float igm = rsqrtf(1.0f + (umx * umx + umy * umy + umz * umz) * a.inv_c2);
  const float tx = kq * f[3] * igm, ty = kq * f[4] * igm, tz = kq * f[5] * igm;
  const float s2 = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
  const float sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
  const float upx = umx + (umy * tz - umz * ty);
  const float upy = umy + (umz * tx - umx * tz);
  const float upz = umz + (umx * ty - umy * tx);
  const float ux = umx + (upy * sz - upz * sy) + kq * f[0];
  const float uy = umy + (upz * sx - upx * sz) + kq * f[1];
  const float uz = umz + (upx * sy - upy * sx) + kq * f[2];
  const float ig = rsqrtf(1.0f + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
  const float vx = ux * ig, vy = uy * ig, vz = uz * ig;
  // displacement in cells
  const float dX = a.dtdx[0] * (vx - a.vg[0]), dY = a.dtdx[1] * (vy - a.vg[1]), dZ = a.dtdx[2] * (vz - a.vg[2]);
  float mfx, mfy, mfz, nfx, nfy, nfz;
  const int mx = ix + move_offset(fx, 0.5f * dX, mfx), my = iy + move_offset(fy, 0.5f * dY, mfy),
            mz = iz + move_offset(fz, 0.5f * dZ, mfz);
  const int nx = ix + move_offset(fx, dX, nfx), ny = iy + move_offset(fy, dY, nfy),
            nz = iz + move_offset(fz, dZ, nfz);
  a.cell[p] = (int)((((int64_t)(nx & a.mask[0]) * a.Ny + (ny & a.mask[1])) * a.Nz) + (nz & a.mask[2]));
  a.fx[p] = nfx;
  a.fy[p] = nfy;
  a.fz[p] = nfz;
  a.ux[p] = ux;
  a.uy[p] = uy;
  a.uz[p] = uz;
  deposit_node_block<P>(a, mx, my, mz, mfx, mfy, mfz, qw * vx, qw * vy, qw * vz, 0.f, true);
  deposit_node_block<P>(a, nx, ny, nz, nfx, nfy, nfz, 0.f, 0.f, 0.f, qw, false);
}

int ilog2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

Push32Args make_args32(pic_ctx* ctx, const pic_species32* sp) {
  Push32Args a;
  a.cell = sp->cell;
  a.fx = sp->fx;
  a.fy = sp->fy;
  a.fz = sp->fz;
  a.ux = sp->ux;
  a.uy = sp->uy;
  a.uz = sp->uz;
  a.w = sp->w;
  a.n = sp->n;
  for (int d = 0; d < 3; ++d) {
    a.mask[d] = (int)ctx->N[d] - 1;
    a.dtdx[d] = (float)(ctx->dt / ctx->dx[d]);
    a.vg[d] = ctx->variant == PIC_PSATD_STANDARD ? 0.0f : (float)ctx->vg[d];
  }
  a.shz = ilog2(ctx->N[2]);
  a.shy = ilog2(ctx->N[1]);
  a.Ny = ctx->N[1];
  a.Nz = ctx->N[2];
  a.qm_half_dt = (float)(sp->q * ctx->dt / (2.0 * sp->m));
  a.inv_c2 = (float)(1.0 / (ctx->c * ctx->c));
  a.qw_scale = (float)(sp->q / (ctx->dx[0] * ctx->dx[1] * ctx->dx[2]));
  return a;
}

pic_status launch_push32(pic_ctx* ctx, const Push32Args& a) {
  if (a.n == 0) return PIC_OK;
  const int bs = 256;
  const unsigned nb = (unsigned)((a.n + bs - 1) / bs);
  switch (ctx->shape_order) {
    case 1: push32_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
    case 2: push32_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
    default: push32_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// tile binning of the FP32 SoA (integer only: tile from the cell index)
// ---------------------------------------------------------------------------
struct Bin32Args {
  const int32_t* cell;
  int64_t n;
  int shz, shy;
  int mask[3];
  int tshift[3];
  int64_t nty, ntz;
  int32_t* tid;
  unsigned long long* counts;
};

__global__ void tile_id32_kernel(Bin32Args a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int c = a.cell[p];
  const int cx = (c >> (a.shz + a.shy)) & a.mask[0], cy = (c >> a.shz) & a.mask[1], cz = c & a.mask[2];
  const int t = (int)(((cx >> a.tshift[0]) * a.nty + (cy >> a.tshift[1])) * a.ntz + (cz >> a.tshift[2]));
  a.tid[p] = t;
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, t);
  const int leader = __ffs(peers) - 1;
  if ((int)(threadIdx.x & 31) == leader) atomicAdd(a.counts + t, (unsigned long long)__popc(peers));
}

__global__ void __launch_bounds__(1024) scan32_kernel(const unsigned long long* cnt, int64_t* off, int64_t n) {
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

struct Scatter32Args {
  const uint32_t* src[9];  // cell, fx, fy, fz, ux, uy, uz, w as 32-bit words
  uint32_t* dst[9];
  const unsigned long long* id_src;
  unsigned long long* id_dst;
  int nfield;
  int64_t n;
  const int32_t* tid;
  const int64_t* off;
  unsigned long long* cursor;
};

__global__ void scatter32_kernel(Scatter32Args a) {
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
  if (a.id_src) a.id_dst[q] = a.id_src[p];
}

}  // namespace

pic_status particles_push32(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                            const pic_species32* sp, float* const J[3], float* rho) {
  Push32Args a = make_args32(ctx, sp);
  for (int c = 0; c < 3; ++c) {
    a.F[c] = En[c];
    a.F[3 + c] = Bn[c];
    a.J[c] = J[c];
  }
  a.rho = rho;
  a.gather = 1;
  return launch_push32(ctx, a);
}

pic_status particles_deposit_rho32(pic_ctx* ctx, const pic_species32* sp, float* rho) {
  Push32Args a = make_args32(ctx, sp);
  for (int c = 0; c < 6; ++c) a.F[c] = nullptr;
  for (int c = 0; c < 3; ++c) a.J[c] = nullptr;
  a.rho = rho;
  a.gather = 0;
  return launch_push32(ctx, a);
}

pic_status particles_bin32(pic_ctx* ctx, const pic_species32* sp, int64_t* offsets_out) {
  const int64_t n = sp->n;
  // scratch: tile ids (int32) and 8 x n 32-bit words + n ids, inside the FP64 binning buffers
  pic_status st = particles_bin_capacity(ctx, n > 0 ? n : 1);
  if (st != PIC_OK) return st;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctx->bin_cursor);
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, ctx->n_tiles * sizeof(int64_t), ctx->stream));
  Bin32Args b;
  b.cell = sp->cell;
  b.n = n;
  b.shz = ilog2(ctx->N[2]);
  b.shy = ilog2(ctx->N[1]);
  for (int d = 0; d < 3; ++d) {
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
    tile_id32_kernel<<<nb, bs, 0, ctx->stream>>>(b);
    PIC_LAUNCH_CHECK(ctx);
  }
  scan32_kernel<<<1, 1024, 0, ctx->stream>>>(cnt, ctx->bin_counts, ctx->n_tiles);
  PIC_LAUNCH_CHECK(ctx);
  if (offsets_out)
    PIC_CUDA_TRY(ctx, cudaMemcpyAsync(offsets_out, ctx->bin_counts, (ctx->n_tiles + 1) * sizeof(int64_t),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
  if (n == 0) return PIC_OK;
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, ctx->n_tiles * sizeof(int64_t), ctx->stream));
  Scatter32Args s;
  void* fields[8] = {sp->cell, sp->fx, sp->fy, sp->fz, sp->ux, sp->uy, sp->uz, sp->w};
  s.nfield = 8;
  uint32_t* tmp = reinterpret_cast<uint32_t*>(ctx->bin_tmp);
  for (int f = 0; f < 8; ++f) {
    s.src[f] = static_cast<const uint32_t*>(fields[f]);
    s.dst[f] = tmp + (int64_t)f * ctx->bin_cap;
  }
  s.id_src = reinterpret_cast<const unsigned long long*>(sp->id);
  s.id_dst = reinterpret_cast<unsigned long long*>(ctx->bin_tmp + 4 * ctx->bin_cap);  // words 8n..10n
  s.n = n;
  s.tid = ctx->bin_tid;
  s.off = ctx->bin_counts;
  s.cursor = cnt;
  scatter32_kernel<<<nb, bs, 0, ctx->stream>>>(s);
  PIC_LAUNCH_CHECK(ctx);
  for (int f = 0; f < 8; ++f)
    PIC_CUDA_TRY(ctx, cudaMemcpyAsync(fields[f], s.dst[f], n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                      ctx->stream));
  if (sp->id)
    PIC_CUDA_TRY(ctx, cudaMemcpyAsync(sp->id, s.id_dst, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  return PIC_OK;
}
