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

#include <algorithm>

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
  int vay;            // 1: Vay's pusher instead of Boris
  // Tiled push only: when src_gate is set and *src_gate != 0 (the binning ran this step), the
  // particles are read from the binning's sorted copy src[0..7] (cell, fx, fy, fz, ux, uy, uz, w
  // as 32-bit words; id_src the ids or null) and written, with w and the ids, to the species
  // arrays: the push is the copy back of the sort.
  const int* src_gate;
  const uint32_t* src[8];
  const unsigned long long* id_src;
  unsigned long long* id_dst;
  float* w_dst;
  // Tiled push only: the species' drift-following tile frame (shift [0..2], velocity [4..6]) and
  // its displacement counters (see particles_frames_advance); null: no frame
  const int* frame;
  unsigned long long* dhist;
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

// u^{n-1/2} = (u0x, u0y, u0z) -> u^{n+1/2} with the gathered f = (E, B): Boris rotation, or Vay's pusher
__device__ __forceinline__ void push_u(const Push32Args& a, float u0x, float u0y, float u0z, const float* f,
                                       float& ux, float& uy, float& uz) {
  const float kq = a.qm_half_dt;
  if (a.vay) {
    ux = u0x;
    uy = u0y;
    uz = u0z;
    vay_push<float>(ux, uy, uz, f, kq, a.inv_c2);
    return;
  }
  const float umx = u0x + kq * f[0], umy = u0y + kq * f[1], umz = u0z + kq * f[2];
  const float igm = rsqrtf(1.0f + (umx * umx + umy * umy + umz * umz) * a.inv_c2);
  const float tx = kq * f[3] * igm, ty = kq * f[4] * igm, tz = kq * f[5] * igm;
  const float s2 = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
  const float sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
  const float upx = umx + (umy * tz - umz * ty);
  const float upy = umy + (umz * tx - umx * tz);
  const float upz = umz + (umx * ty - umy * tx);
  ux = umx + (upy * sz - upz * sy) + kq * f[0];
  uy = umy + (upz * sx - upx * sz) + kq * f[1];
  uz = umz + (upx * sy - upy * sx) + kq * f[2];
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

// Shared-memory deposit window of one tile: nodes [org, org + W) per axis
// (unwrapped coordinates), four fixed-point int32 components (J^x, J^y, J^z, rho;
// value = sum / scale), each [W0][W1][W2] with row stride W2 and plane stride
// `plane` (padded, see TileArgs).
struct Window {
  int* acc;
  int org[3];
  int W[3];
  int plane, comp;
  float sj[3], sr;  // fixed-point scales (powers of two) of the J^x, J^y, J^z and rho sums
};

// Deposit one particle's (P+1)^3 block: inside the window with shared-memory
// integer atomics of the contributions rounded to the window's fixed-point scale,
// outside it (a particle that left its tile since the last binning) with global
// FP32 atomics.  j: (v0, v1, v2) into J, else r into rho.
template <int P>
__device__ __forceinline__ bool deposit_window(const Push32Args& a, const Window& win, int ix, int iy, int iz,
                                               float fx, float fy, float fz, float v0, float v1, float v2, float r,
                                               bool j) {
  constexpr int NS = P + 1;
  int lx, ly, lz;
  float Sx[NS], Sy[NS], Sz[NS];
  shape32<P>(ix, fx, lx, Sx);
  shape32<P>(iy, fy, ly, Sy);
  shape32<P>(iz, fz, lz, Sz);
  // offsets from the window origin modulo N: the (shifted) tile frame may sit across the periodic
  // boundary; a window longer than the grid along an axis holds the same node twice, and either
  // entry flushes to it
  const int wx = (lx - win.org[0]) & a.mask[0], wy = (ly - win.org[1]) & a.mask[1], wz = (lz - win.org[2]) & a.mask[2];
  const bool inside = wx + NS <= win.W[0] && wy + NS <= win.W[1] && wz + NS <= win.W[2];
  if (!inside) {
    // rare (the particle left its tile since the last binning): global atomics, rolled loop
#pragma unroll 1
    for (int i = 0; i < NS; ++i) {
      const int ox = ((lx + i) & a.mask[0]) * (int)a.Ny;
      const float sx = Sx[i];
#pragma unroll
      for (int jj = 0; jj < NS; ++jj) {
        const int oy = (ox + ((ly + jj) & a.mask[1])) * (int)a.Nz;
        const float sxy = sx * Sy[jj];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const int o = oy + ((lz + k) & a.mask[2]);
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
    return false;
  }
  const int comp = win.comp;
  const float w0 = v0 * win.sj[0], w1 = v1 * win.sj[1], w2 = v2 * win.sj[2], wr = r * win.sr;
#pragma unroll(P == 3 ? 1 : NS)
  for (int i = 0; i < NS; ++i) {
#pragma unroll
    for (int jj = 0; jj < NS; ++jj) {
      const float sxy = Sx[i] * Sy[jj];
      int* row = win.acc + (wx + i) * win.plane + (wy + jj) * win.W[2] + wz;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float s = sxy * Sz[k];
        if (j) {
          atomicAdd(row + k, __float2int_rn(s * w0));
          atomicAdd(row + comp + k, __float2int_rn(s * w1));
          atomicAdd(row + 2 * comp + k, __float2int_rn(s * w2));
        } else {
          atomicAdd(row + 3 * comp + k, __float2int_rn(s * wr));
        }
      }
    }
  }
  return true;
}

// z start of a particle's shape block (its first node) relative to its cell
template <int P>
__device__ __forceinline__ int shape_base_offset(float f) {
  return P == 2 ? (f >= 0.5f ? 0 : -1) : (P == 3 ? -1 : 0);
}

// J of one particle (cell (ix, iy, iz) + offsets: the current-deposit midpoint) over NS + 1 z nodes
// from node lz0, its own block starting lz - lz0 = 0 or 1 nodes in and the other node taking 0; a
// particle whose block starts elsewhere, or that leaves the window, deposits through global
// memory.  With lz0 the lowest midpoint block start of the warp relative to the lanes' x^{n+1}
// cells, the lanes address the window relative to those cells, whose pattern fills 32 distinct
// banks: a plasma streaming through a Galilean grid shifts its midpoints by about half a cell,
// which sends neighbouring lanes' per-particle blocks to the same node (bank conflicts that cost
// 6.9 wavefronts per particle on the beam-driven box).  The integer contributions of the block's
// nodes are those of deposit_window.
template <int P>
__device__ __forceinline__ void deposit_j5(const Push32Args& a, const Window& win, int ix, int iy, int iz, float fx,
                                           float fy, float fz, float v0, float v1, float v2, int lz0) {
  constexpr int NS = P + 1;
  int lx, ly, lz;
  float Sx[NS], Sy[NS], Sz[NS];
  shape32<P>(ix, fx, lx, Sx);
  shape32<P>(iy, fy, ly, Sy);
  shape32<P>(iz, fz, lz, Sz);
  const int sh = lz - lz0;
  const int wx = (lx - win.org[0]) & a.mask[0], wy = (ly - win.org[1]) & a.mask[1],
            wz = (lz0 - win.org[2]) & a.mask[2];
  if (!((unsigned)sh <= 1u && wx + NS <= win.W[0] && wy + NS <= win.W[1] && wz + NS + 1 <= win.W[2])) {
#pragma unroll 1
    for (int i = 0; i < NS; ++i) {
      const int ox = ((lx + i) & a.mask[0]) * (int)a.Ny;
      const float sx = Sx[i];
#pragma unroll
      for (int jj = 0; jj < NS; ++jj) {
        const int oy = (ox + ((ly + jj) & a.mask[1])) * (int)a.Nz;
        const float sxy = sx * Sy[jj];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const int o = oy + ((lz + k) & a.mask[2]);
          const float s = sxy * Sz[k];
          atomicAdd(a.J[0] + o, s * v0);
          atomicAdd(a.J[1] + o, s * v1);
          atomicAdd(a.J[2] + o, s * v2);
        }
      }
    }
    return;
  }
  const int comp = win.comp;
  const float w0 = v0 * win.sj[0], w1 = v1 * win.sj[1], w2 = v2 * win.sj[2];
#pragma unroll(P == 3 ? 1 : NS)
  for (int i = 0; i < NS; ++i) {
#pragma unroll
    for (int jj = 0; jj < NS; ++jj) {
      const float sxy = Sx[i] * Sy[jj];
      int* row = win.acc + (wx + i) * win.plane + (wy + jj) * win.W[2] + wz;
#pragma unroll
      for (int k = 0; k <= NS; ++k) {
        const float s = sxy * (sh ? (k > 0 ? Sz[k - 1] : 0.f) : (k < NS ? Sz[k] : 0.f));
        atomicAdd(row + k, __float2int_rn(s * w0));
        atomicAdd(row + comp + k, __float2int_rn(s * w1));
        atomicAdd(row + 2 * comp + k, __float2int_rn(s * w2));
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
  // push u^{n-1/2} -> u^{n+1/2}
  float ux, uy, uz;
  push_u(a, a.ux[p], a.uy[p], a.uz[p], f, ux, uy, uz);
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

// Staggered comparison cycle (Sec. 2), FP32 form: E, B gathered from their own Yee positions,
// J deposited at its Yee positions, rho on the nodes; untiled, global atomics.  On an axis
// staggered by half a cell the shape is taken for (cell, offset) shifted by -1/2:
// offset f >= 1/2 -> (i, f - 1/2), else (i - 1, f + 1/2).
__device__ __forceinline__ void half_shift_cell(int i, float f, int& is, float& fs) {
  if (f >= 0.5f) {
    is = i;
    fs = f - 0.5f;
  } else {
    is = i - 1;
    fs = f + 0.5f;
  }
}

template <int P>
__device__ __forceinline__ float gather32_one(const float* F, const Push32Args& a, const int* lo, const float* Sx,
                                              const float* Sy, const float* Sz) {
  constexpr int NS = P + 1;
  float v = 0.0f;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lo[0] + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((lo[1] + j) & a.mask[1])) * a.Nz;
      const float sxy = Sx[i] * Sy[j];
#pragma unroll
      for (int k = 0; k < NS; ++k) v += sxy * Sz[k] * __ldg(F + oy + ((lo[2] + k) & a.mask[2]));
    }
  }
  return v;
}

template <int P>
__device__ __forceinline__ void deposit32_one(float* F, const Push32Args& a, const int* lo, const float* Sx,
                                              const float* Sy, const float* Sz, float val) {
  constexpr int NS = P + 1;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int64_t ox = (int64_t)((lo[0] + i) & a.mask[0]) * a.Ny;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int64_t oy = (ox + ((lo[1] + j) & a.mask[1])) * a.Nz;
      const float sxy = Sx[i] * Sy[j] * val;
#pragma unroll
      for (int k = 0; k < NS; ++k) atomicAdd(F + oy + ((lo[2] + k) & a.mask[2]), sxy * Sz[k]);
    }
  }
}

// shapes of (cell c[d], offset f[d]) on the nodal (0) and staggered (1) grid of every axis
template <int P>
__device__ __forceinline__ void shapes_both(const int* c, const float* f, int* l0, int* l1, float (*S0)[P + 1],
                                            float (*S1)[P + 1]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    shape32<P>(c[d], f[d], l0[d], S0[d]);
    int is;
    float fs;
    half_shift_cell(c[d], f[d], is, fs);
    shape32<P>(is, fs, l1[d], S1[d]);
  }
}

template <int P>
__global__ void __launch_bounds__(256) push32_stag_kernel(Push32Args a) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  constexpr int NS = P + 1;
  const int cl = a.cell[p];
  const int ci[3] = {(cl >> (a.shz + a.shy)) & a.mask[0], (cl >> a.shz) & a.mask[1], cl & a.mask[2]};
  const float fo[3] = {a.fx[p], a.fy[p], a.fz[p]};
  const float qw = a.w[p] * a.qw_scale;
  int l0[3], l1[3];
  float S0[3][NS], S1[3][NS];
  shapes_both<P>(ci, fo, l0, l1, S0, S1);
  constexpr int kStag[6] = {1, 2, 4, 6, 5, 3};  // Ex, Ey, Ez, Bx, By, Bz
  float f[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int m = kStag[c];
    const int lo[3] = {(m & 1) ? l1[0] : l0[0], (m & 2) ? l1[1] : l0[1], (m & 4) ? l1[2] : l0[2]};
    f[c] = gather32_one<P>(a.F[c], a, lo, (m & 1) ? S1[0] : S0[0], (m & 2) ? S1[1] : S0[1], (m & 4) ? S1[2] : S0[2]);
  }
  float ux, uy, uz;
  push_u(a, a.ux[p], a.uy[p], a.uz[p], f, ux, uy, uz);
  const float ig = rsqrtf(1.0f + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
  const float v[3] = {ux * ig, uy * ig, uz * ig};
  int mc[3], nc[3];
  float mf[3], nf[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float dd = a.dtdx[d] * (v[d] - a.vg[d]);
    mc[d] = ci[d] + move_offset(fo[d], 0.5f * dd, mf[d]);
    nc[d] = ci[d] + move_offset(fo[d], dd, nf[d]);
  }
  a.cell[p] = (((nc[0] & a.mask[0]) * (int)a.Ny + (nc[1] & a.mask[1])) * (int)a.Nz) + (nc[2] & a.mask[2]);
  a.fx[p] = nf[0];
  a.fy[p] = nf[1];
  a.fz[p] = nf[2];
  a.ux[p] = ux;
  a.uy[p] = uy;
  a.uz[p] = uz;
  // J^{n+1/2}: component d at its Yee positions
  shapes_both<P>(mc, mf, l0, l1, S0, S1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int lo[3] = {c == 0 ? l1[0] : l0[0], c == 1 ? l1[1] : l0[1], c == 2 ? l1[2] : l0[2]};
    deposit32_one<P>(a.J[c], a, lo, c == 0 ? S1[0] : S0[0], c == 1 ? S1[1] : S0[1], c == 2 ? S1[2] : S0[2],
                     qw * v[c]);
  }
  // rho^{n+1} on the nodes
#pragma unroll
  for (int d = 0; d < 3; ++d) shape32<P>(nc[d], nf[d], l0[d], S0[d]);
  deposit32_one<P>(a.rho, a, l0, S0[0], S0[1], S0[2], qw);
}

// Tiled form: one CTA per chunk of a particle tile (ranges from the last binning;
// a tile holding more than kTileChunk particles is split into equal chunks so that
// a dense bunch spreads over many SMs).  The tile's nodal E, B plus guard nodes are
// staged in shared memory, J and rho accumulate in a shared-memory window covering
// the tile plus two guard cells on each side (enough for a cubic shape and a move of
// up to one cell), and the window is flushed once with global atomics.
//
// Shared-memory layout.  Binning orders the cells of a tile z fastest, then x, then y,
// so at P particles per cell the 32 lanes of a warp (visiting every P-th particle)
// hold 32 cells: the T2 = 8 z-cells of 4 consecutive x-planes at one y.  Both shared arrays
// are component-planar with the plane stride padded to 8 (mod 32) words, so the
// lanes' addresses for the same relative node fall in 32 distinct banks: every
// gather load and every deposit atomic of such a warp is one conflict-free access.
struct TileArgs {
  const int64_t* off;     // [n_tiles + 1] particle ranges
  const uint32_t* chunk;  // [n_tiles + 1] exclusive prefix sum of chunks per tile
  const uint32_t* chunk_tile;  // tile of each chunk
  int64_t n_tiles;
  unsigned long long* outside;  // count of particles whose new cell left the chunk's tile
  int T[3];               // tile edge (cells)
  int nt[3];              // tiles per axis
  int cpt;                // cells per tile
  int W[3];               // deposit window edge = T + 5
  int wplane, wcomp;      // deposit window plane and component strides (words)
  int G[3];               // gather window edge = T + 3: nodes [T0 - 1, T0 + T + 2)
  int gplane, gcomp;      // gather window plane and component strides (words)
  int vec_flush;          // flush by aligned groups of 4 z nodes (16-byte vector reductions)
};

// threads per chunk CTA: 64 registers each, 4 CTAs per SM (256 threads measured 7% faster than 128)
constexpr int kTileThreads = 256;

// particle of a chunk visited by slot j when every s-th particle goes to consecutive slots
__device__ __forceinline__ int interleaved(int j, int q, int s) {
  const int r = j / q;
  return (j - r * q) * s + r;
}

// phase 2 of the tiled push over the chunk's particles (see push32_tile_kernel)
template <int P, bool JEXT>
__device__ __forceinline__ void deposit_phase(const Push32Args& a, const Window& win, int p0, int cnt, int q, int s) {
  for (int j = threadIdx.x; j < q * s; j += blockDim.x) {
    const int pr = interleaved(j, q, s);
    if (pr >= cnt) continue;
    const int p = p0 + pr;
    const int c = a.cell[p];
    const int nx = (c >> (a.shz + a.shy)) & a.mask[0], ny = (c >> a.shz) & a.mask[1], nz = c & a.mask[2];
    const float nfx = a.fx[p], nfy = a.fy[p], nfz = a.fz[p];
    const float ux = a.ux[p], uy = a.uy[p], uz = a.uz[p];
    const float qw = a.w[p] * a.qw_scale;
    const float ig = rsqrtf(1.0f + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
    const float vx = ux * ig, vy = uy * ig, vz = uz * ig;
    const float hX = -0.5f * a.dtdx[0] * (vx - a.vg[0]), hY = -0.5f * a.dtdx[1] * (vy - a.vg[1]),
                hZ = -0.5f * a.dtdx[2] * (vz - a.vg[2]);
    float mfx, mfy, mfz;
    const int mx = nx + move_offset(nfx, hX, mfx), my = ny + move_offset(nfy, hY, mfy),
              mz = nz + move_offset(nfz, hZ, mfz);
    if (JEXT) {
      const int ozmin = __reduce_min_sync(__activemask(), mz - nz + shape_base_offset<P>(mfz));
      deposit_j5<P>(a, win, mx, my, mz, mfx, mfy, mfz, qw * vx, qw * vy, qw * vz, nz + ozmin);
    } else {
      deposit_window<P>(a, win, mx, my, mz, mfx, mfy, mfz, qw * vx, qw * vy, qw * vz, 0.f, true);
    }
    deposit_window<P>(a, win, nx, ny, nz, nfx, nfy, nfz, 0.f, 0.f, 0.f, qw, false);
  }
}


// JEXT: the J deposit of deposit_phase.  On a grid moving along z a species with a tile frame gets
// both instantiations launched, and the one that does not match its frame's z velocity (nonzero:
// streaming through the grid) returns at once; elsewhere only JEXT = false is launched and runs.
template <int P, bool JEXT>
__global__ void __launch_bounds__(kTileThreads, 1024 / kTileThreads) push32_tile_kernel(Push32Args a, TileArgs t) {
  extern __shared__ float smem[];
  __shared__ int s_tile, s_part;
  __shared__ float s_bnd[4][kTileThreads / 32];
  if (a.vg[2] != 0.0f && (a.frame != nullptr && __ldg(a.frame + 6) != 0) != JEXT) return;
  if (threadIdx.x == 0) {
    // chunk blockIdx.x: its tile from the chunk map, its index within the tile from the chunk starts
    const uint32_t b = blockIdx.x;
    int tl = -1, k = 0;
    if (b < t.chunk[t.n_tiles]) {
      tl = (int)t.chunk_tile[b];
      k = (int)(b - t.chunk[tl]);
    }
    s_tile = tl;
    s_part = k;
  }
  __syncthreads();
  const int tile = s_tile;
  if (tile < 0) return;
  const int tz = tile % t.nt[2], ty = (tile / t.nt[2]) % t.nt[1], tx = tile / (t.nt[1] * t.nt[2]);
  // the tile's cells start at tile * T + the species' frame shift (0 without a frame); the next push
  // sees the frame moved by its velocity
  __shared__ int s_next[3];  // first cell of the tile in the next push's frame, per axis
  int fs[3] = {0, 0, 0};
  if (a.frame) {
#pragma unroll
    for (int d = 0; d < 3; ++d) fs[d] = __ldg(a.frame + d);
  }
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    const int tc = d == 0 ? tx : (d == 1 ? ty : tz);
    const int sh = d == 0 ? fs[0] : (d == 1 ? fs[1] : fs[2]);
    const int te = d == 0 ? t.T[0] : (d == 1 ? t.T[1] : t.T[2]);
    s_next[d] = tc * te + sh + (a.frame ? __ldg(a.frame + 4 + d) : 0);
  }
  Window win;
  win.org[0] = tx * t.T[0] - 2 + fs[0];
  win.org[1] = ty * t.T[1] - 2 + fs[1];
  win.org[2] = tz * t.T[2] - 2 + fs[2];
  for (int d = 0; d < 3; ++d) win.W[d] = t.W[d];
  win.plane = t.wplane;
  win.comp = t.wcomp;
  win.acc = reinterpret_cast<int*>(smem);
  const int G1 = t.G[1], G2 = t.G[2], gplane = t.gplane, gcomp = t.gcomp;
  // the staged fields are needed in phase 1 only and the deposit window in phase 2 only:
  // both live at the start of the dynamic shared memory
  // [3][G0][G1][G2] pairs (E_x, E_y), (E_z, B_x), (B_y, B_z), plane stride gplane: one 8-byte load
  // reads two components of a node
  float2* fld = reinterpret_cast<float2*>(smem);
  const int go0 = tx * t.T[0] - 1 + fs[0], go1 = ty * t.T[1] - 1 + fs[1], go2 = tz * t.T[2] - 1 + fs[2];
  int p0, cnt, ppc;
  {
    const int64_t b0 = t.off[tile], cnt_t = t.off[tile + 1] - b0;
    const int64_t nch = t.chunk[tile + 1] - t.chunk[tile], k = s_part;
    p0 = (int)(b0 + cnt_t * k / nch);
    cnt = (int)(b0 + cnt_t * (k + 1) / nch) - p0;
    ppc = (int)min((int64_t)cnt, (cnt_t + (t.cpt >> 1)) / t.cpt);  // particles per cell of the tile
  }
  const int gvol = t.G[0] * G1 * G2;
  for (int e = threadIdx.x; e < gvol; e += blockDim.x) {
    const int k = e % G2, r = e / G2;
    const int j = r % G1, i = r / G1;
    const int o = (((go0 + i) & a.mask[0]) * (int)a.Ny + ((go1 + j) & a.mask[1])) * (int)a.Nz + ((go2 + k) & a.mask[2]);
    const int d = i * gplane + j * G2 + k;
#pragma unroll
    for (int q = 0; q < 3; ++q) fld[q * gcomp + d] = make_float2(__ldg(a.F[2 * q] + o), __ldg(a.F[2 * q + 1] + o));
  }
  __syncthreads();
  constexpr int NS = P + 1;
  // visit every s-th particle (s ~ the tile's particles per cell) so that a warp's lanes hold
  // distinct cells; a chunk of a dense tile spans only cnt / s cells, and its lanes spread over them
  const int s = max(1, ppc);
  const int q = (cnt + s - 1) / s;
  unsigned nout = 0;
  // Phase 1: gather, Boris push and move of every particle of the chunk; the new state goes to
  // memory.  Each thread sums |q w v_c| (c = x, y, z) and |q w| over its particles.
  float bnd[4] = {0.f, 0.f, 0.f, 0.f};
  // per thread: counts of the cell displacements -1 and +1 per axis in 5-bit fields (a thread
  // visits at most ceil(2048 / 256) + 1 particles of its chunk)
  unsigned dpk = 0u;
  const bool sorted_src = a.src_gate != nullptr && *a.src_gate != 0;
  for (int j = threadIdx.x; j < q * s; j += blockDim.x) {
    const int pr = interleaved(j, q, s);
    if (pr >= cnt) continue;
    const int p = p0 + pr;
    int c;
    float fx, fy, fz, u0x, u0y, u0z, wp;
    if (sorted_src) {
      c = (int)a.src[0][p];
      fx = __uint_as_float(a.src[1][p]);
      fy = __uint_as_float(a.src[2][p]);
      fz = __uint_as_float(a.src[3][p]);
      u0x = __uint_as_float(a.src[4][p]);
      u0y = __uint_as_float(a.src[5][p]);
      u0z = __uint_as_float(a.src[6][p]);
      wp = __uint_as_float(a.src[7][p]);
      a.w_dst[p] = wp;
      if (a.id_src) a.id_dst[p] = a.id_src[p];
    } else {
      c = a.cell[p];
      fx = a.fx[p];
      fy = a.fy[p];
      fz = a.fz[p];
      u0x = a.ux[p];
      u0y = a.uy[p];
      u0z = a.uz[p];
      wp = a.w[p];
    }
    const int ix = (c >> (a.shz + a.shy)) & a.mask[0], iy = (c >> a.shz) & a.mask[1], iz = c & a.mask[2];
    int lx, ly, lz;
    float Sx[NS], Sy[NS], Sz[NS];
    shape32<P>(ix, fx, lx, Sx);
    shape32<P>(iy, fy, ly, Sy);
    shape32<P>(iz, fz, lz, Sz);
    float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int gx = (lx - go0) & a.mask[0], gy = (ly - go1) & a.mask[1], gz = (lz - go2) & a.mask[2];
    const bool gin = gx + NS <= t.G[0] && gy + NS <= G1 && gz + NS <= G2;
    if (gin) {
      // cubic: the outer loop stays rolled (a 4x smaller hot loop for the instruction cache,
      // measured 6% faster together with the deposit loop); lower orders fully unrolled
#pragma unroll(P == 3 ? 1 : NS)
      for (int i = 0; i < NS; ++i) {
#pragma unroll
        for (int jj = 0; jj < NS; ++jj) {
          const float sxy = Sx[i] * Sy[jj];
          const float2* row = fld + (gx + i) * gplane + (gy + jj) * G2 + gz;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const float w = sxy * Sz[k];
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
              const float2 v = row[qq * gcomp + k];
              f[2 * qq] += w * v.x;
              f[2 * qq + 1] += w * v.y;
            }
          }
        }
      }
    } else {
      // rare (the particle left its tile since the last binning): kept rolled to keep the
      // kernel's hot loop compact in the instruction cache
#pragma unroll 1
      for (int i = 0; i < NS; ++i) {
        const int ox = ((lx + i) & a.mask[0]) * (int)a.Ny;
        const float sx = Sx[i];
#pragma unroll
        for (int jj = 0; jj < NS; ++jj) {
          const int oy = (ox + ((ly + jj) & a.mask[1])) * (int)a.Nz;
          const float sxy = sx * Sy[jj];
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const int o = oy + ((lz + k) & a.mask[2]);
            const float w = sxy * Sz[k];
#pragma unroll
            for (int qq = 0; qq < 6; ++qq) f[qq] += w * __ldg(a.F[qq] + o);
          }
        }
      }
    }
    float ux, uy, uz;
    push_u(a, u0x, u0y, u0z, f, ux, uy, uz);
    const float ig = rsqrtf(1.0f + (ux * ux + uy * uy + uz * uz) * a.inv_c2);
    const float vx = ux * ig, vy = uy * ig, vz = uz * ig;
    const float dX = a.dtdx[0] * (vx - a.vg[0]), dY = a.dtdx[1] * (vy - a.vg[1]), dZ = a.dtdx[2] * (vz - a.vg[2]);
    float nfx, nfy, nfz;
    const int nx = ix + move_offset(fx, dX, nfx), ny = iy + move_offset(fy, dY, nfy),
              nz = iz + move_offset(fz, dZ, nfz);
    // the next push gathers this particle from the staged nodes of this tile only while its new
    // cell stays in the tile: count those that leave (the device re-bins before the next push
    // when they exceed 2 % of all particles)
    nout += (((nx - s_next[0]) & a.mask[0]) >= t.T[0] || ((ny - s_next[1]) & a.mask[1]) >= t.T[1] ||
             ((nz - s_next[2]) & a.mask[2]) >= t.T[2])
                ? 1u
                : 0u;
    // cell displacements -1 and +1 per axis (the frame velocity estimate of the next step)
    dpk += (nx - ix == -1 ? 1u : 0u) + (nx - ix == 1 ? 1u << 5 : 0u) + (ny - iy == -1 ? 1u << 10 : 0u) +
           (ny - iy == 1 ? 1u << 15 : 0u) + (nz - iz == -1 ? 1u << 20 : 0u) + (nz - iz == 1 ? 1u << 25 : 0u);
    a.cell[p] = (((nx & a.mask[0]) * (int)a.Ny + (ny & a.mask[1])) * (int)a.Nz) + (nz & a.mask[2]);
    a.fx[p] = nfx;
    a.fy[p] = nfy;
    a.fz[p] = nfz;
    a.ux[p] = ux;
    a.uy[p] = uy;
    a.uz[p] = uz;
    const float qw = fabsf(wp * a.qw_scale);
    bnd[0] += qw * fabsf(vx);
    bnd[1] += qw * fabsf(vy);
    bnd[2] += qw * fabsf(vz);
    bnd[3] += qw;
  }
  // Fixed-point scales.  A node sum of component c is at most S_max^3 sum_p |q w v_c| (J) or
  // S_max^3 sum_p |q w| (rho), S_max the largest 1D shape weight; each scale is the power of
  // two that puts this bound below 2^30, so the int32 sums (plus at most 1/2 per rounded
  // contribution) cannot overflow, and every contribution is rounded to 2^-30 of the chunk's
  // own bound: the window sums are exact integers, independent of the atomic order.
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bnd[c] += __shfl_xor_sync(0xffffffffu, bnd[c], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) s_bnd[c][threadIdx.x >> 5] = bnd[c];
  }
  __syncthreads();
  float scale[4];
  {
    const float smax3 = P == 1 ? 1.0f : (P == 2 ? 0.421875f : 0.2962963f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float b = 0.0f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_bnd[c][w];
      b *= smax3 * 1.001f;  // margin for the rounding of the sums and of S_max^3
      // b < 2^(ilogb(b) + 1), so b * 2^(29 - ilogb(b)) < 2^30
      scale[c] = b > 0.0f ? ldexpf(1.0f, min(126, max(-126, 29 - ilogbf(b)))) : 1.0f;
    }
  }
  win.sj[0] = scale[0];
  win.sj[1] = scale[1];
  win.sj[2] = scale[2];
  win.sr = scale[3];
  // the staged fields are dead: clear the deposit window in their place
  // (4 wcomp floats, wcomp a multiple of 8: 16-byte stores)
  for (int e = threadIdx.x; e < t.wcomp; e += blockDim.x)
    reinterpret_cast<float4*>(smem)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  // Phase 2: deposit J^{n+1/2} at the midpoint x^{n+1} - (dt/2)(v - v_gal) and rho^{n+1} at
  // x^{n+1}, from the state written in phase 1 (same thread, same particles).  A species whose
  // tile frame streams along z (frame velocity != 0: the particles cross a cell per step relative
  // to the grid) deposits J over NS + 1 z nodes from the warp's lowest midpoint block
  // (deposit_j5), the others one block per particle.
  deposit_phase<P, JEXT>(a, win, p0, cnt, q, s);
  nout = __reduce_add_sync(0xffffffffu, nout);
  if (nout && (threadIdx.x & 31) == 0) atomicAdd(t.outside, (unsigned long long)nout);
  if (a.dhist) {
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const unsigned c = __reduce_add_sync(0xffffffffu, (dpk >> (5 * e)) & 31u);
      if (c && (threadIdx.x & 31) == 0) atomicAdd(a.dhist + e, (unsigned long long)c);
    }
  }
  __syncthreads();
  // flush the window: node (i, j, k) of the window is global node org + (i, j, k), wrapped
  float* dst[4] = {a.J[0], a.J[1], a.J[2], a.rho};
  float inv[4];  // exact: the scales are powers of two
#pragma unroll
  for (int c = 0; c < 4; ++c) inv[c] = 1.0f / scale[c];
  const int W1 = t.W[1], W2 = t.W[2];
  if (t.vec_flush) {
    // Window rows along z cover nodes [org, org + W2); they are flushed as the aligned groups of 4
    // nodes starting at org rounded down to a multiple of 4 (Nz is a multiple of 4, so a group
    // never wraps), one 16-byte vector reduction per group and component, nodes outside the window
    // adding 0, groups whose four sums are all 0 skipped: about a third of the scalar reductions.
    const int z0 = win.org[2] & ~3;
    const int nq = (win.org[2] - z0 + W2 + 3) >> 2;
    const int vol4 = t.W[0] * W1 * nq;
    for (int e = threadIdx.x; e < vol4; e += blockDim.x) {
      const int g = e % nq, r = e / nq;
      const int j = r % W1, i = r / W1;
      const int k0 = z0 + 4 * g - win.org[2];  // window index of the group's first node
      const int o = (((win.org[0] + i) & a.mask[0]) * (int)a.Ny + ((win.org[1] + j) & a.mask[1])) * (int)a.Nz +
                    ((win.org[2] + k0) & a.mask[2]);
      const int d = i * t.wplane + j * W2 + k0;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        int iv[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) iv[l] = (k0 + l >= 0 && k0 + l < W2) ? win.acc[qq * t.wcomp + d + l] : 0;
        if ((iv[0] | iv[1] | iv[2] | iv[3]) != 0)
          atomicAdd(reinterpret_cast<float4*>(dst[qq] + o),
                    make_float4((float)iv[0] * inv[qq], (float)iv[1] * inv[qq], (float)iv[2] * inv[qq],
                                (float)iv[3] * inv[qq]));
      }
    }
    return;
  }
  const int vol = t.W[0] * W1 * W2;
  for (int e = threadIdx.x; e < vol; e += blockDim.x) {
    const int k = e % W2, r = e / W2;
    const int j = r % W1, i = r / W1;
    const int o = (((win.org[0] + i) & a.mask[0]) * (int)a.Ny + ((win.org[1] + j) & a.mask[1])) * (int)a.Nz +
                  ((win.org[2] + k) & a.mask[2]);
    const int d = i * t.wplane + j * W2 + k;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const int iv = win.acc[qq * t.wcomp + d];
      if (iv != 0) atomicAdd(dst[qq] + o, (float)iv * inv[qq]);
    }
  }
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
  a.vay = ctx->pusher == PIC_PUSHER_VAY ? 1 : 0;
  a.qw_scale = (float)(sp->q / (ctx->dx[0] * ctx->dx[1] * ctx->dx[2]));
  a.src_gate = nullptr;
  for (int f = 0; f < 8; ++f) a.src[f] = nullptr;
  a.id_src = nullptr;
  a.id_dst = nullptr;
  a.w_dst = nullptr;
  a.frame = nullptr;
  a.dhist = nullptr;
  return a;
}

pic_status launch_push32(pic_ctx* ctx, const Push32Args& a) {
  if (a.n == 0) return PIC_OK;
  const int bs = 256;
  const unsigned nb = (unsigned)((a.n + bs - 1) / bs);
  if (a.gather && ctx->cycle == PIC_CYCLE_STAGGERED) {
    switch (ctx->shape_order) {
      case 1: push32_stag_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
      case 2: push32_stag_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
      default: push32_stag_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
    }
    PIC_LAUNCH_CHECK(ctx);
    return PIC_OK;
  }
  switch (ctx->shape_order) {
    case 1: push32_kernel<1><<<nb, bs, 0, ctx->stream>>>(a); break;
    case 2: push32_kernel<2><<<nb, bs, 0, ctx->stream>>>(a); break;
    default: push32_kernel<3><<<nb, bs, 0, ctx->stream>>>(a); break;
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

// elements scanned per block by the multi-block exclusive scan of the binning
constexpr int kScanBlock = 4096;

// start of the chunk -> tile map inside a chunk list
size_t chunk_map_offset(const pic_ctx* ctx) {
  return (size_t)ctx->n_tiles + 1 + (size_t)((ctx->n_tiles + kScanBlock - 1) / kScanBlock) + 1;
}

// smallest stride >= v that is 8 or 24 (mod 32) words: a warp's lanes (8 z cells x 4 x planes)
// then fall on 32 distinct banks (z + 8 x or z + 24 x, mod 32)
int pad_plane(int v) {
  const int a = v + (((8 - v) % 32) + 32) % 32, b = v + (((24 - v) % 32) + 32) % 32;
  return std::min(a, b);
}

// tile geometry and shared-memory strides of the tiled push; returns the dynamic shared bytes.
// The window spans the tile, 2 nodes before it and 3 after it on every axis (the cubic block of a
// particle one cell past the tile), except 2 after it along x when wx_after = 2 (see
// launch_push32_tiled): a particle that moved past the tile's upper x face since its binning then
// deposits through global memory.
size_t tile_layout(const pic_ctx* ctx, TileArgs& t, int wx_after) {
  t.cpt = 1;
  for (int d = 0; d < 3; ++d) {
    t.T[d] = ctx->tile[d];
    t.nt[d] = (int)(ctx->N[d] / ctx->tile[d]);
    t.W[d] = ctx->tile[d] + (d == 0 ? 2 + wx_after : 5);
    t.G[d] = ctx->tile[d] + 3;
    t.cpt *= ctx->tile[d];
  }
  t.wplane = pad_plane(t.W[1] * t.W[2]);
  t.wcomp = t.W[0] * t.wplane;
  t.gplane = pad_plane(t.G[1] * t.G[2]);
  t.gcomp = t.G[0] * t.gplane;
  return std::max(4 * (size_t)t.wcomp, 6 * (size_t)t.gcomp) * sizeof(float);
}

pic_status launch_push32_tiled(pic_ctx* ctx, const Push32Args& a, const int64_t* off, const uint32_t* chunk) {
  if (a.n == 0) return PIC_OK;
  TileArgs t;
  t.off = off;
  t.chunk = chunk;
  t.chunk_tile = chunk + chunk_map_offset(ctx);
  t.n_tiles = ctx->n_tiles;
  t.outside = ctx->bin_outside;
  // the window one node shorter along x when that lets more CTAs share an SM (e.g. 8 x 16 x 8
  // tiles: 3 -> 4 CTAs, the register limit)
  size_t smem = tile_layout(ctx, t, 3);
  {
    TileArgs t2 = t;
    const size_t smem2 = tile_layout(ctx, t2, 2);
    const void* fn = ctx->shape_order == 1 ? (const void*)push32_tile_kernel<1, false>
                     : ctx->shape_order == 2 ? (const void*)push32_tile_kernel<2, false>
                                             : (const void*)push32_tile_kernel<3, false>;
    const void* fx = ctx->shape_order == 1 ? (const void*)push32_tile_kernel<1, true>
                     : ctx->shape_order == 2 ? (const void*)push32_tile_kernel<2, true>
                                             : (const void*)push32_tile_kernel<3, true>;
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int n3 = 0, n2 = 0;
    PIC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n3, fn, kTileThreads, smem));
    PIC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, fn, kTileThreads, smem2));
    if (n2 > n3) {
      t = t2;
      smem = smem2;
    }
  }
  bool aligned = ctx->N[2] % 4 == 0;
  const float* dsts[4] = {a.J[0], a.J[1], a.J[2], a.rho};
  for (const float* d : dsts) aligned = aligned && (reinterpret_cast<uintptr_t>(d) % 16 == 0);
  t.vec_flush = aligned ? 1 : 0;
  // sum over tiles of ceil(count / kTileChunk) < n_tiles + n / kTileChunk: surplus CTAs return at once
  const unsigned nb = (unsigned)(ctx->n_tiles + (a.n + kTileChunk - 1) / kTileChunk);
  switch (ctx->shape_order) {
    case 1: push32_tile_kernel<1, false><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
    case 2: push32_tile_kernel<2, false><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
    default: push32_tile_kernel<3, false><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
  }
  PIC_LAUNCH_CHECK(ctx);
  // the twin only on a grid moving along z (v_gal_z != 0), where a plasma at rest streams through
  // the grid; elsewhere a species with a z frame velocity takes the per-particle J blocks of the
  // first launch
  if (a.frame != nullptr && a.vg[2] != 0.0f) {
    switch (ctx->shape_order) {
      case 1: push32_tile_kernel<1, true><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
      case 2: push32_tile_kernel<2, true><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
      default: push32_tile_kernel<3, true><<<nb, kTileThreads, smem, ctx->stream>>>(a, t); break;
    }
    PIC_LAUNCH_CHECK(ctx);
  }
  return PIC_OK;
}

// ---------------------------------------------------------------------------
// binning of the FP32 SoA: counting sort by cell in tile-major order
// key = tile * cells_per_tile + local cell (z fastest, then x, then y), so particles end up grouped by
// tile and, inside a tile, ordered by cell (integer only: from the cell index)
// ---------------------------------------------------------------------------
// Binning runs only when *gate is non-zero (the device decides, see bin_decide_kernel), so it can
// be enqueued every step without a host round trip.
__device__ __forceinline__ bool gated_off(const int* gate) { return gate != nullptr && *gate == 0; }

__global__ void fill_u32_kernel(uint32_t* p, int64_t n, uint32_t v, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

// scatter gate = binning gate (1 without one) && the keys were out of order: an already sorted
// species needs its tile ranges but no permutation
__global__ void scatter_gate_kernel(const int* gate, const int* unsorted, int* sgate) {
  *sgate = ((gate == nullptr || *gate != 0) && *unsorted != 0) ? 1 : 0;
}

// gate = (particles whose new cell left their tile in the last push) > limit, or forced; resets the count
__global__ void bin_decide_kernel(int* gate, unsigned long long* outside, unsigned long long limit, int force) {
  *gate = (force || *outside > limit) ? 1 : 0;
  *outside = 0ull;
}

struct FrameArgs {
  int* frame;                 // + 8 q: shift [0..2], velocity [4..6]
  unsigned long long* dhist;  // + 10 q: counts of displacements -1, +1 for x, y, z
  int64_t n[PIC_MAX_BINNED_SPECIES];
  int mask[3];
  int nsp;
};

// one thread per species: the frame moves by the velocity the last push assumed; the new velocity
// is the displacement at least 3/4 of the species' particles made (else 0)
__global__ void frames_advance_kernel(FrameArgs a) {
  const int q = threadIdx.x;
  if (q >= a.nsp) return;
  int* f = a.frame + 8 * q;
  unsigned long long* h = a.dhist + 10 * q;
  const unsigned long long n = (unsigned long long)a.n[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d] = (f[d] + f[4 + d]) & a.mask[d];
    const unsigned long long neg = h[2 * d], pos = h[2 * d + 1];
    f[4 + d] = (n > 0 && 4 * neg >= 3 * n) ? -1 : ((n > 0 && 4 * pos >= 3 * n) ? 1 : 0);
    h[2 * d] = 0ull;
    h[2 * d + 1] = 0ull;
  }
}

struct Key32Args {
  const int* gate;
  const int32_t* cell;
  int64_t n;
  int shz, shy;
  int mask[3];
  int tshift[3];
  int tmask[3];
  int64_t nty, ntz;
  int lshift_x, lshift_z;  // log2 of the tile edge in x, z (local cell index: z fastest, then x, then y)
  int cpt_shift;           // log2 cells per tile
  int32_t* key;
  uint32_t* counts;
  int* unsorted;           // set to 1 when some key is smaller than its predecessor's
  const int* frame;        // the species' tile frame (shift at [0..2]) or null
  int sh[3];               // its shift, loaded by each kernel (load_frame)
};

// the tile frame's shift into the kernel's copy of the arguments (0 without a frame)
__device__ __forceinline__ Key32Args load_frame(const Key32Args& a) {
  Key32Args k = a;
#pragma unroll
  for (int d = 0; d < 3; ++d) k.sh[d] = a.frame ? __ldg(a.frame + d) : 0;
  return k;
}

// key of a cell: tile of the cell shifted by -sh (the tile frame), then the local cell inside it
__device__ __forceinline__ int key_of(const Key32Args& a, int c) {
  const int cx = ((c >> (a.shz + a.shy)) - a.sh[0]) & a.mask[0], cy = ((c >> a.shz) - a.sh[1]) & a.mask[1],
            cz = (c - a.sh[2]) & a.mask[2];
  const int t = (int)(((cx >> a.tshift[0]) * a.nty + (cy >> a.tshift[1])) * a.ntz + (cz >> a.tshift[2]));
  const int local = ((((cy & a.tmask[1]) << a.lshift_x) | (cx & a.tmask[0])) << a.lshift_z) | (cz & a.tmask[2]);
  return (t << a.cpt_shift) | local;
}

__device__ __forceinline__ bool key32_one(const Key32Args& a, int64_t p) {
  const int k = key_of(a, a.cell[p]);
  a.key[p] = k;
  const unsigned active = __activemask();
  // already in key order?  (the lanes of a warp hold consecutive particles; lane 0 reads its
  // predecessor's cell)
  const int lane_id = threadIdx.x & 31;
  const int up = __shfl_up_sync(active, k, 1);
  const int prev = lane_id > 0 ? up : (p > 0 ? key_of(a, a.cell[p - 1]) : k);
  const unsigned peers = __match_any_sync(active, k);
  const int leader = __ffs(peers) - 1;
  if ((int)(threadIdx.x & 31) == leader) atomicAdd(a.counts + k, (uint32_t)__popc(peers));
  return prev > k;
}

// "some key is smaller than its predecessor's": one global store per block at most (a store per
// out-of-order particle to the same word serialises at L2 when many particles moved)
__device__ __forceinline__ void flag_unsorted(const Key32Args& a, bool mine) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  if (mine) s_any = 1;
  __syncthreads();
  if (threadIdx.x == 0 && s_any) *a.unsorted = 1;
}

__global__ void key32_kernel(Key32Args a0) {
  if (gated_off(a0.gate)) return;
  const Key32Args a = load_frame(a0);
  bool mine = false;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x)
    mine |= key32_one(a, p);
  flag_unsorted(a, mine);
}

// exclusive scan, phase 1: each block scans 4096 counts in place (to offsets within the block)
// and writes its total to bsum[block]
__device__ __forceinline__ void scan_one_block(uint32_t* v, int64_t n, uint32_t* bsum, int64_t blk,
                                               uint32_t* part) {
  const int64_t base = blk * kScanBlock;
  uint32_t x[4];
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + threadIdx.x * 4 + q;
    x[q] = i < n ? v[i] : 0u;
    s += x[q];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const uint32_t t = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + threadIdx.x * 4 + q;
    if (i < n) v[i] = run;
    run += x[q];
  }
  if (threadIdx.x == 1023) bsum[blk] = part[1023];
}

__global__ void __launch_bounds__(1024) scan_block_kernel(uint32_t* v, int64_t n, uint32_t* bsum, const int* gate) {
  if (gated_off(gate)) return;
  __shared__ uint32_t part[1024];
  const int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    __syncthreads();  // part[] of the previous block is consumed
    scan_one_block(v, n, bsum, blk, part);
  }
}

// phase 2: one CTA scans the block totals (exclusive) and writes the grand total
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t* bsum, int64_t nb, uint32_t* total,
                                                         const int* gate) {
  if (gated_off(gate)) return;
  __shared__ uint32_t part[1024];
  const int64_t chunk = (nb + 1023) / 1024;
  const int64_t b = threadIdx.x * chunk, e = min(nb, b + chunk);
  uint32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += bsum[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const uint32_t t = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
  for (int64_t i = b; i < e; ++i) {
    const uint32_t c = bsum[i];
    bsum[i] = run;
    run += c;
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

// phase 3: add the block offsets; also emit the per-tile ranges off[t] = cell offset of the tile's first key
__global__ void scan_add_kernel(uint32_t* v, int64_t n, const uint32_t* bsum, int cpt_shift, int64_t* tile_off,
                                int64_t n_tiles, const uint32_t* total, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = v[i] + bsum[i / kScanBlock];
    v[i] = o;
    if ((i & ((int64_t(1) << cpt_shift) - 1)) == 0) tile_off[i >> cpt_shift] = (int64_t)o;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_off[n_tiles] = (int64_t)*total;
}

// map[k] = tile of chunk k, for the chunks [start[t], start[t + 1]) of every tile t
__global__ void chunk_map_kernel(const uint32_t* start, int64_t n_tiles, uint32_t* map, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles; t += (int64_t)gridDim.x * blockDim.x)
    for (uint32_t k = start[t]; k < start[t + 1]; ++k) map[k] = (uint32_t)t;
}

// chunks per tile: nch[t] = ceil(count_t / kTileChunk), scanned in place afterwards
__global__ void chunk_count_kernel(const int64_t* off, int64_t n_tiles, uint32_t* nch, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_tiles; i += (int64_t)gridDim.x * blockDim.x)
    nch[i] = (uint32_t)((off[i + 1] - off[i] + kTileChunk - 1) / kTileChunk);
}

__global__ void chunk_add_kernel(uint32_t* v, int64_t n, const uint32_t* bsum, const uint32_t* total,
                                 const int* gate) {
  if (gated_off(gate)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] += bsum[i / kScanBlock];
  if (i == 0) v[n] = *total;
}

struct Scatter32Args {
  const int* gate;
  const uint32_t* src[8];  // cell, fx, fy, fz, ux, uy, uz, w as 32-bit words
  uint32_t* dst[8];
  const unsigned long long* id_src;
  unsigned long long* id_dst;
  int64_t n;
  const int32_t* key;
  const uint32_t* off;     // exclusive offsets per key
  uint32_t* cursor;        // zeroed
};

__device__ __forceinline__ void scatter32_one(const Scatter32Args& a, int64_t p);

__global__ void scatter32_kernel(Scatter32Args a) {
  if (gated_off(a.gate)) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x)
    scatter32_one(a, p);
}

__device__ __forceinline__ void scatter32_one(const Scatter32Args& a, int64_t p) {
  const int k = a.key[p];
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, k);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(a.cursor + k, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int64_t q = (int64_t)a.off[k] + base + rank;
#pragma unroll
  for (int f = 0; f < 8; ++f) a.dst[f][q] = a.src[f][p];
  if (a.id_src) a.id_dst[q] = a.id_src[p];
}

// copy the sorted scratch back into the species arrays (8 words + optional id per particle); used by
// pic_bin32 only: inside pic_step32 the next tiled push reads the sorted copy instead
struct CopyBackArgs {
  const int* gate;
  const uint32_t* src[8];
  uint32_t* dst[8];
  const unsigned long long* id_src;
  unsigned long long* id_dst;
  int64_t n;
};

__global__ void copy_back_kernel(CopyBackArgs a) {
  if (gated_off(a.gate)) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int f = 0; f < 8; ++f) a.dst[f][p] = a.src[f][p];
    if (a.id_src) a.id_dst[p] = a.id_src[p];
  }
}

// ---------------------------------------------------------------------------
// two-level binning (tiles whose cells fit the shared-memory ordering, <= kMaxLocalCells)
// level 1: counting sort by tile.  The particles arrive nearly in key order (binned before the
//   last push, which moves them by about a cell), so the 32 lanes of a warp fall in one or two
//   tiles: counts and cursors take one atomic per tile per warp (__match_any_sync), and the tile
//   offsets come from a scan over the tiles only (no per-cell passes).
// level 2: one CTA per tile orders the tile's particles by local cell (z fastest, then x, then y)
//   with a shared-memory counting sort and writes them back into the species arrays.
// ---------------------------------------------------------------------------
constexpr int kMaxLocalCells = 4096;
constexpr int kOrderThreads = 256;

// per particle: key (sortedness check against its predecessor) and the tile histogram
__global__ void tile_count_kernel(Key32Args a0) {
  if (gated_off(a0.gate)) return;
  const Key32Args a = load_frame(a0);
  bool mine = false;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int k = key_of(a, a.cell[p]);
    const unsigned active = __activemask();
    const int lane_id = threadIdx.x & 31;
    const int up = __shfl_up_sync(active, k, 1);
    const int prev = lane_id > 0 ? up : (p > 0 ? key_of(a, a.cell[p - 1]) : k);
    mine |= prev > k;
    const int t = k >> a.cpt_shift;
    const unsigned peers = __match_any_sync(active, t);
    if (lane_id == __ffs(peers) - 1) atomicAdd(a.counts + t, (uint32_t)__popc(peers));
  }
  flag_unsorted(a, mine);
}

struct TileScatterArgs {
  const int* gate;
  Key32Args k;
  uint32_t* spc[8];                // the species arrays: cell, fx, fy, fz, ux, uy, uz, w as 32-bit words
  uint32_t* tmp[8];                // scratch of the same layout
  unsigned long long* id_spc;      // optional ids
  unsigned long long* id_tmp;
  const uint32_t* off;             // exclusive tile offsets
  uint32_t* cursor;                // zeroed, per tile
};

// level 1: species arrays -> scratch, grouped by tile (order inside a tile: arbitrary)
__global__ void tile_scatter_kernel(TileScatterArgs a) {
  if (gated_off(a.gate)) return;
  a.k = load_frame(a.k);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.k.n; p += (int64_t)gridDim.x * blockDim.x) {
    // the particle's words are loaded before the cursor atomic (which the compiler may not move
    // them past), so their latency overlaps it
    uint32_t v[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) v[f] = a.spc[f][p];
    const unsigned long long id = a.id_spc ? a.id_spc[p] : 0ull;
    const int t = key_of(a.k, (int)v[0]) >> a.k.cpt_shift;
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, t);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(a.cursor + t, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t q = (int64_t)a.off[t] + base + rank;
#pragma unroll
    for (int f = 0; f < 8; ++f) a.tmp[f][q] = v[f];
    if (a.id_spc) a.id_tmp[q] = id;
  }
}

// level 2: scratch -> species arrays, each tile ordered by local cell: one CTA per tile (grid-stride
// over the tiles), a shared-memory counting sort (the order among the particles of one cell is
// that of the shared-memory atomics, i.e. unspecified)
__global__ void __launch_bounds__(kOrderThreads) cell_order_kernel(TileScatterArgs a, const int64_t* tile_off,
                                                                   int64_t n_tiles) {
  if (gated_off(a.gate)) return;
  a.k = load_frame(a.k);
  __shared__ uint32_t cnt[kMaxLocalCells];
  __shared__ uint32_t part[kOrderThreads];
  const int cpt = 1 << a.k.cpt_shift;
  const int lmask = cpt - 1;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t b0 = tile_off[t], nt = tile_off[t + 1] - b0;
    if (nt == 0) continue;  // uniform over the CTA
    for (int i = threadIdx.x; i < cpt; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nt; i += blockDim.x)
      atomicAdd(&cnt[key_of(a.k, (int)a.tmp[0][b0 + i]) & lmask], 1u);
    __syncthreads();
    // exclusive scan of cnt[0..cpt): each thread a run of cpt / blockDim entries
    const int per = (cpt + blockDim.x - 1) / blockDim.x;
    const int i0 = min(cpt, (int)threadIdx.x * per), i1 = min(cpt, i0 + per);
    uint32_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {
      const uint32_t v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
    for (int i = i0; i < i1; ++i) {
      const uint32_t c = cnt[i];
      cnt[i] = run;
      run += c;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) {
      const int64_t j = b0 + i;
      uint32_t v[8];
#pragma unroll
      for (int f = 0; f < 8; ++f) v[f] = a.tmp[f][j];
      const unsigned long long id = a.id_spc ? a.id_tmp[j] : 0ull;
      const int l = key_of(a.k, (int)v[0]) & lmask;
      const int64_t q = b0 + atomicAdd(&cnt[l], 1u);
#pragma unroll
      for (int f = 0; f < 8; ++f) a.spc[f][q] = v[f];
      if (a.id_spc) a.id_spc[q] = id;
    }
    __syncthreads();  // cnt is reused by the next tile
  }
}

}  // namespace

#ifndef PIC_BIN_LIMIT
#define PIC_BIN_LIMIT 0.02
#endif

pic_status particles_bin32_decide(pic_ctx* ctx, int64_t total_particles, int force) {
  const unsigned long long limit = (unsigned long long)(PIC_BIN_LIMIT * (double)total_particles);
  bin_decide_kernel<<<1, 1, 0, ctx->stream>>>(ctx->bin_gate, ctx->bin_outside, limit, force);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status particles_frames_advance(pic_ctx* ctx, const pic_species32* sp, int n_species) {
  FrameArgs f;
  f.frame = ctx->frame;
  f.dhist = ctx->dhist;
  f.nsp = std::min(n_species, PIC_MAX_BINNED_SPECIES);
  for (int q = 0; q < PIC_MAX_BINNED_SPECIES; ++q) f.n[q] = q < f.nsp ? sp[q].n : 0;
  for (int d = 0; d < 3; ++d) f.mask[d] = (int)ctx->N[d] - 1;
  if (f.nsp <= 0 || !ctx->frame) return PIC_OK;
  frames_advance_kernel<<<1, 32, 0, ctx->stream>>>(f);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

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

bool bin32_two_level(const pic_ctx* ctx) {
  return int64_t(ctx->tile[0]) * ctx->tile[1] * ctx->tile[2] <= kMaxLocalCells;
}

int bin32_launches(const pic_ctx* ctx, int64_t n, bool chunks, bool copy_back) {
  // fill, (count), three scan kernels, (five chunk-list kernels), then for n > 0 the scatter gate,
  // the cursor fill and the scatter (and the in-tile ordering, or the copy back)
  const int head = 1 + (n > 0 ? 1 : 0) + 3 + (chunks ? 5 : 0);
  if (n == 0) return head;
  return head + 3 + ((bin32_two_level(ctx) || copy_back) ? 1 : 0);
}

bool tiled_push_fits(const pic_ctx* ctx) {
  TileArgs t;
  return tile_layout(ctx, t, 3) <= 160 * 1024 && ctx->ncell < (int64_t(1) << 31);
}

size_t tile_chunk_words(const pic_ctx* ctx, int64_t n) {
  // chunk starts [n_tiles + 1], scan block sums, scan total, tile of each chunk
  return chunk_map_offset(ctx) + (size_t)ctx->n_tiles + (size_t)(n / kTileChunk) + 1;
}

pic_status particles_push32_tiled(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                                  const pic_species32* sp, float* const J[3], float* rho, const int64_t* offsets,
                                  const uint32_t* chunks, const int* sorted_gate, const int* frame,
                                  unsigned long long* dhist) {
  Push32Args a = make_args32(ctx, sp);
  a.frame = frame;
  a.dhist = dhist;
  for (int c = 0; c < 3; ++c) {
    a.F[c] = En[c];
    a.F[3 + c] = Bn[c];
    a.J[c] = J[c];
  }
  a.rho = rho;
  a.gather = 1;
  if (sorted_gate) {
    // the binning of this species (if the gate let it run) left its sorted copy in bin_tmp
    const uint32_t* tmp = reinterpret_cast<const uint32_t*>(ctx->bin_tmp);
    a.src_gate = sorted_gate;
    for (int f = 0; f < 8; ++f) a.src[f] = tmp + (int64_t)f * ctx->bin_cap;
    a.id_src = sp->id ? reinterpret_cast<const unsigned long long*>(ctx->bin_tmp + 4 * ctx->bin_cap) : nullptr;
    a.id_dst = reinterpret_cast<unsigned long long*>(sp->id);
    a.w_dst = sp->w;
  }
  return launch_push32_tiled(ctx, a, offsets, chunks);
}

pic_status particles_deposit_rho32(pic_ctx* ctx, const pic_species32* sp, float* rho) {
  Push32Args a = make_args32(ctx, sp);
  for (int c = 0; c < 6; ++c) a.F[c] = nullptr;
  for (int c = 0; c < 3; ++c) a.J[c] = nullptr;
  a.rho = rho;
  a.gather = 0;
  return launch_push32(ctx, a);
}

// chunk list of the tiled push from the tile ranges: chunks per tile, their exclusive scan and the
// chunk -> tile map (see particles_push32_tiled)
static pic_status build_chunks(pic_ctx* ctx, const int64_t* tile_off, uint32_t* chunks_out, const int* gate) {
  const int64_t nt = ctx->n_tiles;
  const int64_t nblk_t = (nt + kScanBlock - 1) / kScanBlock;
  const unsigned fill_blocks = 152 * 8;
  uint32_t* cbsum = chunks_out + nt + 1;
  uint32_t* ctotal = cbsum + nblk_t;
  chunk_count_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(tile_off, nt, chunks_out, gate);
  PIC_LAUNCH_CHECK(ctx);
  scan_block_kernel<<<(unsigned)std::min<int64_t>(nblk_t, 152 * 2), 1024, 0, ctx->stream>>>(chunks_out, nt, cbsum,
                                                                                          gate);
  PIC_LAUNCH_CHECK(ctx);
  scan_sums_kernel<<<1, 1024, 0, ctx->stream>>>(cbsum, nblk_t, ctotal, gate);
  PIC_LAUNCH_CHECK(ctx);
  chunk_add_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(chunks_out, nt, cbsum, ctotal, gate);
  PIC_LAUNCH_CHECK(ctx);
  chunk_map_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(chunks_out, nt, chunks_out + chunk_map_offset(ctx), gate);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status particles_bin32(pic_ctx* ctx, const pic_species32* sp, int64_t* offsets_out, const int* gate,
                           uint32_t* chunks_out, bool copy_back, const int* frame) {
  const int64_t n = sp->n;
  pic_status st = particles_bin_capacity(ctx, n > 0 ? n : 1);
  if (st != PIC_OK) return st;
  const int64_t ncell = ctx->ncell;
  const int64_t nblk = (ncell + kScanBlock - 1) / kScanBlock;
  if (!ctx->cell_counts) {
    // counts/offsets per cell, block sums, total
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->cell_counts, (ncell + nblk + 2) * sizeof(uint32_t)));
  }
  uint32_t* counts = ctx->cell_counts;
  uint32_t* bsum = counts + ncell;
  uint32_t* total = bsum + nblk;
  const unsigned fill_blocks = 152 * 8;
  Key32Args b;
  b.gate = gate;
  b.cell = sp->cell;
  b.n = n;
  b.shz = ilog2(ctx->N[2]);
  b.shy = ilog2(ctx->N[1]);
  for (int d = 0; d < 3; ++d) {
    b.mask[d] = (int)ctx->N[d] - 1;
    b.tshift[d] = ilog2(ctx->tile[d]);
    b.tmask[d] = ctx->tile[d] - 1;
  }
  b.nty = ctx->N[1] / ctx->tile[1];
  b.ntz = ctx->N[2] / ctx->tile[2];
  b.lshift_x = ilog2(ctx->tile[0]);
  b.lshift_z = ilog2(ctx->tile[2]);
  b.cpt_shift = ilog2(ctx->tile[0]) + ilog2(ctx->tile[1]) + ilog2(ctx->tile[2]);
  b.key = ctx->bin_tid;
  b.counts = counts;
  b.frame = frame;
  b.sh[0] = b.sh[1] = b.sh[2] = 0;
  if (!ctx->bin_flags) PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->bin_flags, 2 * sizeof(int)));
  int* unsorted = ctx->bin_flags;
  int* sgate = ctx->bin_flags + 1;
  b.unsorted = unsorted;
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(unsorted, 0, sizeof(int), ctx->stream));
  // grid-stride kernels on a capped grid: when the gate is off they return at once, so a gated
  // binning costs a few microseconds, not a full-size launch
  const int bs = 256;
  const unsigned nb = (unsigned)std::min<int64_t>((n + bs - 1) / bs, fill_blocks);
  int64_t* tile_off = offsets_out ? offsets_out : ctx->bin_counts;
  if ((int64_t(1) << b.cpt_shift) <= kMaxLocalCells) {
    // two-level: counting sort by tile, then by cell inside each tile (see tile_count_kernel)
    const int64_t nt = ctx->n_tiles;
    const int64_t nblk_t = (nt + kScanBlock - 1) / kScanBlock;
    uint32_t* tcnt = counts;           // per tile: counts -> exclusive offsets
    uint32_t* tbsum = counts + nt;     // scan block sums
    uint32_t* ttotal = tbsum + nblk_t;
    fill_u32_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(tcnt, nt, 0u, gate);
    PIC_LAUNCH_CHECK(ctx);
    if (n > 0) {
      tile_count_kernel<<<nb, bs, 0, ctx->stream>>>(b);
      PIC_LAUNCH_CHECK(ctx);
    }
    scan_block_kernel<<<(unsigned)std::min<int64_t>(nblk_t, 152 * 2), 1024, 0, ctx->stream>>>(tcnt, nt, tbsum, gate);
    PIC_LAUNCH_CHECK(ctx);
    scan_sums_kernel<<<1, 1024, 0, ctx->stream>>>(tbsum, nblk_t, ttotal, gate);
    PIC_LAUNCH_CHECK(ctx);
    scan_add_kernel<<<(unsigned)std::min<int64_t>((nt + 255) / 256, fill_blocks), 256, 0, ctx->stream>>>(
        tcnt, nt, tbsum, 0, tile_off, nt, ttotal, gate);
    PIC_LAUNCH_CHECK(ctx);
    if (chunks_out) PIC_TRY(build_chunks(ctx, tile_off, chunks_out, gate));
    if (n == 0) {
      PIC_CUDA_TRY(ctx, cudaMemsetAsync(sgate, 0, sizeof(int), ctx->stream));
      return PIC_OK;
    }
    scatter_gate_kernel<<<1, 1, 0, ctx->stream>>>(gate, unsorted, sgate);
    PIC_LAUNCH_CHECK(ctx);
    if (!ctx->cell_cursor) PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->cell_cursor, ncell * sizeof(uint32_t)));
    fill_u32_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(ctx->cell_cursor, nt, 0u, sgate);
    PIC_LAUNCH_CHECK(ctx);
    TileScatterArgs s;
    s.gate = sgate;
    s.k = b;
    void* fields[8] = {sp->cell, sp->fx, sp->fy, sp->fz, sp->ux, sp->uy, sp->uz, sp->w};
    uint32_t* tmp = reinterpret_cast<uint32_t*>(ctx->bin_tmp);
    for (int f = 0; f < 8; ++f) {
      s.spc[f] = static_cast<uint32_t*>(fields[f]);
      s.tmp[f] = tmp + (int64_t)f * ctx->bin_cap;
    }
    s.id_spc = reinterpret_cast<unsigned long long*>(sp->id);
    s.id_tmp = reinterpret_cast<unsigned long long*>(ctx->bin_tmp + 4 * ctx->bin_cap);  // words 8n..10n
    s.off = tcnt;
    s.cursor = ctx->cell_cursor;
    tile_scatter_kernel<<<nb, bs, 0, ctx->stream>>>(s);
    PIC_LAUNCH_CHECK(ctx);
    cell_order_kernel<<<(unsigned)std::min<int64_t>(nt, 152 * 8), kOrderThreads, 0, ctx->stream>>>(s, tile_off, nt);
    PIC_LAUNCH_CHECK(ctx);
    return PIC_OK;  // the species arrays hold the binned particles
  }
  // one level: counting sort by cell in tile-major order over the whole grid
  fill_u32_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(counts, ncell, 0u, gate);
  PIC_LAUNCH_CHECK(ctx);
  if (n > 0) {
    key32_kernel<<<nb, bs, 0, ctx->stream>>>(b);
    PIC_LAUNCH_CHECK(ctx);
  }
  scan_block_kernel<<<(unsigned)std::min<int64_t>(nblk, 152 * 2), 1024, 0, ctx->stream>>>(counts, ncell, bsum, gate);
  PIC_LAUNCH_CHECK(ctx);
  scan_sums_kernel<<<1, 1024, 0, ctx->stream>>>(bsum, nblk, total, gate);
  PIC_LAUNCH_CHECK(ctx);
  scan_add_kernel<<<(unsigned)std::min<int64_t>((ncell + 255) / 256, fill_blocks), 256, 0, ctx->stream>>>(
      counts, ncell, bsum, b.cpt_shift, tile_off, ctx->n_tiles, total, gate);
  PIC_LAUNCH_CHECK(ctx);
  if (chunks_out) PIC_TRY(build_chunks(ctx, tile_off, chunks_out, gate));
  if (n == 0) {
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(sgate, 0, sizeof(int), ctx->stream));
    return PIC_OK;
  }
  scatter_gate_kernel<<<1, 1, 0, ctx->stream>>>(gate, unsorted, sgate);
  PIC_LAUNCH_CHECK(ctx);
  if (!ctx->cell_cursor) PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->cell_cursor, ncell * sizeof(uint32_t)));
  fill_u32_kernel<<<fill_blocks, 256, 0, ctx->stream>>>(ctx->cell_cursor, ncell, 0u, sgate);
  PIC_LAUNCH_CHECK(ctx);
  Scatter32Args s;
  s.gate = sgate;
  void* fields[8] = {sp->cell, sp->fx, sp->fy, sp->fz, sp->ux, sp->uy, sp->uz, sp->w};
  uint32_t* tmp = reinterpret_cast<uint32_t*>(ctx->bin_tmp);
  for (int f = 0; f < 8; ++f) {
    s.src[f] = static_cast<const uint32_t*>(fields[f]);
    s.dst[f] = tmp + (int64_t)f * ctx->bin_cap;
  }
  s.id_src = reinterpret_cast<const unsigned long long*>(sp->id);
  s.id_dst = reinterpret_cast<unsigned long long*>(ctx->bin_tmp + 4 * ctx->bin_cap);  // words 8n..10n
  s.n = n;
  s.key = ctx->bin_tid;
  s.off = counts;
  s.cursor = ctx->cell_cursor;
  scatter32_kernel<<<nb, bs, 0, ctx->stream>>>(s);
  PIC_LAUNCH_CHECK(ctx);
  if (!copy_back) return PIC_OK;  // the next tiled push reads the sorted copy
  CopyBackArgs cb;
  cb.gate = sgate;
  for (int f = 0; f < 8; ++f) {
    cb.src[f] = s.dst[f];
    cb.dst[f] = static_cast<uint32_t*>(fields[f]);
  }
  cb.id_src = sp->id ? s.id_dst : nullptr;
  cb.id_dst = reinterpret_cast<unsigned long long*>(sp->id);
  cb.n = n;
  copy_back_kernel<<<152 * 8, 256, 0, ctx->stream>>>(cb);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}
