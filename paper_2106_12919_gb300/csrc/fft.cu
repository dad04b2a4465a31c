// 3D real-to-complex FFT for the PSATD solver: shared-memory Stockham kernels,
// templated on the precision (FP64 form: double; FP32 form: float).
//
// Forward: z-axis R2C (a length-Nz/2 complex FFT of packed (even, odd) pairs
// followed by the split step), then in-place C2C along y and along x.
// Inverse: C2C along x, along y, then z-axis C2R.  Plain DFT, unnormalised:
// X_m = sum_j x_j exp(-2 pi i j.m / N) (App. A.1, Eq. Fourier_discrete without
// the half-cell phase, which the caller applies).
//
// Every CTA transforms a whole tile of lines: radix-8 (+ one radix-4 or radix-2) Stockham passes
// with every length a template parameter (one kernel per power of two, all index arithmetic
// compile-time shifts and masks).  Pass 0 takes its butterfly's inputs straight from global memory
// into registers, the last pass of a C2C or C2R transform writes straight back, so a transform of
// npass passes goes through shared memory npass - 1 times.  z lines are contiguous (line-major
// tile, padded one slot per 16 elements to spread the radix-8 scatter over the banks); y and x
// lines are strided, so a CTA takes W adjacent columns (consecutive k_z) and the tile is
// element-major, which keeps the global loads coalesced in W-element rows.  The passes read their
// twiddles from per-pass tables (fft_tile.cuh).  In the FP32 form the z passes run as persistent
// kernels whose next tile arrives by a bulk copy while the current one is transformed.
#include "pic_internal.cuh"
#include "fft_tile.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kZTile = 2048;             // complex elements per z-pass CTA (L lines * Nz/2)
constexpr int kZThreads = kZTile / 8;    // one radix-8 butterfly per thread

using namespace pic_fft;

// z-axis real-to-complex: L = 4096 / M lines of Nz = 2M reals -> M + 1 complex per line.  Each
// thread loads its pass-0 butterfly (8 packed (even, odd) pairs, stride M / 8) straight from global
// memory.
template <class T, int LGM>
__global__ void __launch_bounds__(kZThreads, (sizeof(T) == 4 ? 1536 : 1024) / kZThreads)
    fft_z_r2c_kernel(CRP6<T> in, CP6<typename Cplx<T>::type> out, int64_t nlines,
                     const typename Cplx<T>::type* __restrict__ tw, const typename Cplx<T>::type* __restrict__ twp) {
  using C = typename Cplx<T>::type;
  constexpr int M = 1 << LGM, L = kZTile / M, lgnb = LGM - 3, nb = 1 << lgnb;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  {
    const int l = threadIdx.x >> lgnb, j = threadIdx.x & (nb - 1);
    const int64_t line = line0 + l;
    const C* src = reinterpret_cast<const C*>(in.p[comp]) + line * M + j;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = line < nlines ? src[r * nb] : czero<C>();
    pass0_from_regs<false>(sm, lay, v, j, l);
  }
  passes_ct<false, LGM, 1, Plan<LGM>::npass>(sm, lay, twp);
  // split: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W^k (Z_k - conj Z_{M-k}),  W = exp(-2 pi i / Nz)
  C* dst = out.p[comp];
  constexpr int nzh = M + 1, lgH = LGM - 1;
  const T h = (T)0.5;
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  for (int t = threadIdx.x; t < (L << lgH) + L; t += blockDim.x) {
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    const int64_t line = line0 + l;
    if (line >= nlines) continue;
    const C Zk = sm[lay.idx(k, l)];
    const C Zm = sm[lay.idx((M - k) & (M - 1), l)];
    C Fe, Fo;
    Fe.x = h * (Zk.x + Zm.x);
    Fe.y = h * (Zk.y - Zm.y);
    Fo.x = h * (Zk.y + Zm.y);
    Fo.y = -h * (Zk.x - Zm.x);
    const C wFo = cmul(__ldg(&tw[k]), Fo);
    C* o = dst + line * nzh;
    o[k] = cadd(Fe, wFo);
    if (k != M - k) o[M - k] = cconj(csub(Fe, wFo));
  }
}

// z-axis complex-to-real (unnormalised inverse); the imaginary parts of X_0, X_{Nz/2} are ignored.
// The last pass writes its outputs straight to global memory.
template <class T, int LGM>
__global__ void __launch_bounds__(kZThreads, (sizeof(T) == 4 ? 1536 : 1024) / kZThreads)
    fft_z_c2r_kernel(CP6<typename Cplx<T>::type> in, RP6<T> out, int64_t nlines,
                     const typename Cplx<T>::type* __restrict__ tw, const typename Cplx<T>::type* __restrict__ twp) {
  using C = typename Cplx<T>::type;
  constexpr int M = 1 << LGM, L = kZTile / M;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const C* srcb = in.p[comp];
  constexpr int nzh = M + 1, P = M / 2 + 1, lgH = LGM - 1;
  // Z_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  constexpr int kBatch = (L * P + kZThreads - 1) / kZThreads;
  C xk[kBatch], xm[kBatch];
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const int t = threadIdx.x + q * kZThreads;
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    const int64_t line = line0 + l;
    xk[q] = xm[q] = czero<C>();
    if (t < L * P && line < nlines) {
      xk[q] = srcb[line * nzh + k];
      xm[q] = srcb[line * nzh + (M - k)];
    }
  }
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const int t = threadIdx.x + q * kZThreads;
    if (t >= L * P) break;
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    C Xk = xk[q], Xm = xm[q];
    if (k == 0) {
      Xk.y = 0;
      Xm.y = 0;
    }
    C A, D;
    A.x = Xk.x + Xm.x;
    A.y = Xk.y - Xm.y;
    D.x = Xk.x - Xm.x;
    D.y = Xk.y + Xm.y;
    const C w = __ldg(&tw[k]);
    sm[lay.idx(k, l)] = cadd(A, cmuli(cmul(cconj(w), D)));
    if (k != 0 && k != M - k) sm[lay.idx(M - k, l)] = cadd(cconj(A), cmuli(cmul(w, cconj(D))));
  }
  __syncthreads();
  passes_ct<true, LGM, 0, Plan<LGM>::npass - 1>(sm, lay, twp);
  C* dst = reinterpret_cast<C*>(out.p[comp]) + line0 * M;
  const int nvalid = (int)min((int64_t)L, nlines - line0);
  last_pass_to<true, LGM>(sm, lay, twp, [&](int l, int e, C v) {
    if (l < nvalid) dst[l * M + e] = v;
  });
}

// ---------------------------------------------------------------------------
// Persistent FP32 z passes: a CTA walks over tiles t = blockIdx.x + i gridDim.x (every component's
// tiles in turn) with a staging buffer in shared memory that one bulk copy (cp.async.bulk) fills
// with the next tile's contiguous input while the CTA transforms the current one.  The copy
// completes on an mbarrier whose waits are bounded: a wait that gives up sets the error flag (read
// back by pic_sync as PIC_ERR_TIMEOUT), waits again (bounded) for the copy still in flight and
// returns.
// ---------------------------------------------------------------------------
constexpr int kZPipeCtasPerSm = 1536 / kZThreads;

struct ZPipe {
  int64_t nlines;
  int tiles_per_comp, ntiles;
  int* err;
};

// issue the bulk copy of tile t's input (lines of `line_elems` elements of C) into the staging buffer
template <class C, int L>
__device__ __forceinline__ void zpipe_issue(const ZPipe& zp, const C* const* src, int line_elems, int t, C* stage,
                                            uint64_t* bar) {
  const int comp = t / zp.tiles_per_comp;
  const int64_t line0 = (int64_t)(t - comp * zp.tiles_per_comp) * L;
  const int nvalid = (int)min((int64_t)L, zp.nlines - line0);
  const uint32_t bytes = (uint32_t)nvalid * line_elems * (uint32_t)sizeof(C);
  fence_proxy_async_shared();  // the CTA's earlier reads of the buffer come before the copy's writes
  mbar_arrive_expect_tx(bar, bytes);
  bulk_load(stage, src[comp] + line0 * line_elems, bytes, bar);
}

// wait for the staging buffer's i-th fill; false (after recording the timeout) when it gave up
__device__ __forceinline__ bool zpipe_wait(uint64_t* bar, int i, int* err) {
  const bool ok = mbar_wait_bounded(bar, (uint32_t)(i & 1));
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    mbar_wait_bounded(bar, (uint32_t)(i & 1));  // the copy still in flight lands before the CTA leaves
    return false;
  }
  return true;
}

template <int LGM>
__global__ void __launch_bounds__(kZThreads, kZPipeCtasPerSm)
    fft_z_r2c_pipe_kernel(CRP6<float> in, CP6<float2> out, ZPipe zp, const float2* __restrict__ tw,
                          const float2* __restrict__ twp) {
  using C = float2;
  constexpr int M = 1 << LGM, L = kZTile / M, lgnb = LGM - 3, nb = 1 << lgnb;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bar;
  C* stage = reinterpret_cast<C*>(smraw);  // L lines x M, contiguous
  C* sm = stage + L * M;                    // working tile, padded lines
  const LayLine lay{zline_len(M)};
  const C* const* src = reinterpret_cast<const C* const*>(in.p);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if ((int)blockIdx.x < zp.ntiles) zpipe_issue<C, L>(zp, src, M, blockIdx.x, stage, &bar);
  }
  __syncthreads();
  const int l0 = threadIdx.x >> lgnb, j0 = threadIdx.x & (nb - 1);
  int i = 0;
  for (int t = blockIdx.x; t < zp.ntiles; t += gridDim.x, ++i) {
    const int comp = t / zp.tiles_per_comp;
    const int64_t line0 = (int64_t)(t - comp * zp.tiles_per_comp) * L;
    if (!zpipe_wait(&bar, i, zp.err)) return;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = stage[l0 * M + j0 + r * nb];  // lines past the end: never stored
    __syncthreads();  // the staging buffer is free: fetch the next tile behind this one's passes
    if (threadIdx.x == 0 && t + (int)gridDim.x < zp.ntiles) zpipe_issue<C, L>(zp, src, M, t + gridDim.x, stage, &bar);
    pass0_from_regs<false>(sm, lay, v, j0, l0);
    passes_ct<false, LGM, 1, Plan<LGM>::npass>(sm, lay, twp);
    // split: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W^k (Z_k - conj Z_{M-k}),  W = exp(-2 pi i / Nz)
    C* dst = out.p[comp];
    constexpr int nzh = M + 1, lgH = LGM - 1;
    for (int u = threadIdx.x; u < (L << lgH) + L; u += blockDim.x) {
      const bool mid = u >= (L << lgH);
      const int l = mid ? u - (L << lgH) : u >> lgH;
      const int k = mid ? (M >> 1) : u & ((M >> 1) - 1);
      const int64_t line = line0 + l;
      if (line >= zp.nlines) continue;
      const C Zk = sm[lay.idx(k, l)];
      const C Zm = sm[lay.idx((M - k) & (M - 1), l)];
      C Fe, Fo;
      Fe.x = 0.5f * (Zk.x + Zm.x);
      Fe.y = 0.5f * (Zk.y - Zm.y);
      Fo.x = 0.5f * (Zk.y + Zm.y);
      Fo.y = -0.5f * (Zk.x - Zm.x);
      const C wFo = cmul(__ldg(&tw[k]), Fo);
      C* o = dst + line * nzh;
      o[k] = cadd(Fe, wFo);
      if (k != M - k) o[M - k] = cconj(csub(Fe, wFo));
    }
    __syncthreads();  // the working tile is read before the next tile's pass 0 writes it
  }
}

template <int LGM>
__global__ void __launch_bounds__(kZThreads, kZPipeCtasPerSm)
    fft_z_c2r_pipe_kernel(CP6<float2> in, RP6<float> out, ZPipe zp, const float2* __restrict__ tw,
                          const float2* __restrict__ twp) {
  using C = float2;
  constexpr int M = 1 << LGM, L = kZTile / M, nzh = M + 1, P = M / 2 + 1, lgH = LGM - 1;
  constexpr int kBatch = (L * P + kZThreads - 1) / kZThreads;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bar;
  C* stage = reinterpret_cast<C*>(smraw);            // L lines x (M + 1), contiguous
  C* sm = stage + ((L * nzh + 1) & ~1);              // working tile, padded lines (16-byte aligned)
  const LayLine lay{zline_len(M)};
  const C* const* src = in.p;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if ((int)blockIdx.x < zp.ntiles) zpipe_issue<C, L>(zp, src, nzh, blockIdx.x, stage, &bar);
  }
  __syncthreads();
  int i = 0;
  for (int t = blockIdx.x; t < zp.ntiles; t += gridDim.x, ++i) {
    const int comp = t / zp.tiles_per_comp;
    const int64_t line0 = (int64_t)(t - comp * zp.tiles_per_comp) * L;
    const int nvalid = (int)min((int64_t)L, zp.nlines - line0);
    if (!zpipe_wait(&bar, i, zp.err)) return;
    // Z_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
    // k = 0 .. M/2 - 1 for every line (u < L M / 2), then k = M/2 (u >= L M / 2)
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const int u = threadIdx.x + q * kZThreads;
      if (u >= L * P) break;
      const bool mid = u >= (L << lgH);
      const int l = mid ? u - (L << lgH) : u >> lgH;
      const int k = mid ? (M >> 1) : u & ((M >> 1) - 1);
      C Xk = czero<C>(), Xm = czero<C>();
      if (l < nvalid) {
        Xk = stage[l * nzh + k];
        Xm = stage[l * nzh + M - k];
      }
      if (k == 0) {
        Xk.y = 0;
        Xm.y = 0;
      }
      C A, D;
      A.x = Xk.x + Xm.x;
      A.y = Xk.y - Xm.y;
      D.x = Xk.x - Xm.x;
      D.y = Xk.y + Xm.y;
      const C w = __ldg(&tw[k]);
      sm[lay.idx(k, l)] = cadd(A, cmuli(cmul(cconj(w), D)));
      if (k != 0 && k != M - k) sm[lay.idx(M - k, l)] = cadd(cconj(A), cmuli(cmul(w, cconj(D))));
    }
    __syncthreads();  // the staging buffer is free: fetch the next tile behind this one's passes
    if (threadIdx.x == 0 && t + (int)gridDim.x < zp.ntiles) zpipe_issue<C, L>(zp, src, nzh, t + gridDim.x, stage, &bar);
    passes_ct<true, LGM, 0, Plan<LGM>::npass - 1>(sm, lay, twp);
    float2* dst = reinterpret_cast<float2*>(out.p[comp]) + line0 * M;
    last_pass_to<true, LGM>(sm, lay, twp, [&](int l, int e, C v) {
      if (l < nvalid) dst[l * M + e] = v;
    });
    __syncthreads();  // the working tile is read before the next tile's pre-processing writes it
  }
}

// In-place C2C of length N = 2^LGN along a strided axis: element e of column col of outer line o
// of component c at p[c] + o * os + e * es + col.  A CTA takes W = 2^LGW adjacent columns
// (element-major tile, rows of W elements coalesced); pass 0 takes its inputs from global memory
// and the last pass writes back to it.
// resident CTAs per SM the register cap is set for: ~1280 threads (FP32, 48 registers) or 1024 (FP64, 64)
template <int T, int C_BYTES>
struct StridedMinBlocks {
  static constexpr int raw = (C_BYTES == 16 ? 1024 : 1536) / T;
  static constexpr int value = raw < 1 ? 1 : (raw > 16 ? 16 : raw);
};

template <bool INV, class C, int LGN, int LGW>
__global__ void __launch_bounds__((1 << (LGN + LGW)) / 8, (StridedMinBlocks<(1 << (LGN + LGW)) / 8, sizeof(C)>::value))
    fft_strided_kernel(CP6<C> data, int64_t es, int64_t os, int ncols, const C* __restrict__ twp) {
  constexpr int N = 1 << LGN, W = 1 << LGW, nb = N / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayCol lay{LGW};
  const int comp = blockIdx.z;
  const int col0 = blockIdx.x * W;
  C* base = data.p[comp] + (int64_t)blockIdx.y * os + col0;
  const int wv = min(W, ncols - col0);
  const int w = threadIdx.x & (W - 1), j = threadIdx.x >> LGW;
  C v[8];
  {
    const C* src = base + j * es + w;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = w < wv ? src[r * nb * es] : czero<C>();
  }
  if constexpr (LGN == 3) {  // one radix-8 pass: registers to global memory
    dft<8, INV>(v);
    if (w < wv) {
#pragma unroll
      for (int r = 0; r < 8; ++r) base[r * es + w] = v[r];
    }
  } else {
    pass0_from_regs<INV>(sm, lay, v, j, w);
    passes_ct<INV, LGN, 1, Plan<LGN>::npass - 1>(sm, lay, twp);
    last_pass_to<INV, LGN>(sm, lay, twp, [&](int l, int e, C val) {
      if (l < wv) base[e * es + l] = val;
    });
  }
}

// log2 of the columns per CTA of the strided passes (measured: 16 and 8 equal, 32 slower)
constexpr int strided_lgw(int lgN) { return lgN >= 10 ? 3 : 4; }

template <class C>
using StridedFn = void (*)(CP6<C>, int64_t, int64_t, int, const C*);

template <bool INV, class C, int LGN>
StridedFn<C> strided_at() {
  return fft_strided_kernel<INV, C, LGN, strided_lgw(LGN)>;
}

// the kernel for N = 2^lgN (8 <= N <= 1024)
template <bool INV, class C>
StridedFn<C> strided_fn(int lgN) {
  switch (lgN) {
    case 3: return strided_at<INV, C, 3>();
    case 4: return strided_at<INV, C, 4>();
    case 5: return strided_at<INV, C, 5>();
    case 6: return strided_at<INV, C, 6>();
    case 7: return strided_at<INV, C, 7>();
    case 8: return strided_at<INV, C, 8>();
    case 9: return strided_at<INV, C, 9>();
    case 10: return strided_at<INV, C, 10>();
  }
  return nullptr;
}

template <class T>
using ZR2CFn = void (*)(CRP6<T>, CP6<typename Cplx<T>::type>, int64_t, const typename Cplx<T>::type*,
                        const typename Cplx<T>::type*);
template <class T>
using ZC2RFn = void (*)(CP6<typename Cplx<T>::type>, RP6<T>, int64_t, const typename Cplx<T>::type*,
                        const typename Cplx<T>::type*);

// the z kernels for M = Nz / 2 = 2^lgM (8 <= M <= 512)
template <class T>
ZR2CFn<T> z_r2c_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_r2c_kernel<T, 3>;
    case 4: return fft_z_r2c_kernel<T, 4>;
    case 5: return fft_z_r2c_kernel<T, 5>;
    case 6: return fft_z_r2c_kernel<T, 6>;
    case 7: return fft_z_r2c_kernel<T, 7>;
    case 8: return fft_z_r2c_kernel<T, 8>;
    case 9: return fft_z_r2c_kernel<T, 9>;
  }
  return nullptr;
}
template <class T>
ZC2RFn<T> z_c2r_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_c2r_kernel<T, 3>;
    case 4: return fft_z_c2r_kernel<T, 4>;
    case 5: return fft_z_c2r_kernel<T, 5>;
    case 6: return fft_z_c2r_kernel<T, 6>;
    case 7: return fft_z_c2r_kernel<T, 7>;
    case 8: return fft_z_c2r_kernel<T, 8>;
    case 9: return fft_z_c2r_kernel<T, 9>;
  }
  return nullptr;
}

using ZR2CPipeFn = void (*)(CRP6<float>, CP6<float2>, ZPipe, const float2*, const float2*);
using ZC2RPipeFn = void (*)(CP6<float2>, RP6<float>, ZPipe, const float2*, const float2*);

ZR2CPipeFn z_r2c_pipe_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_r2c_pipe_kernel<3>;
    case 4: return fft_z_r2c_pipe_kernel<4>;
    case 5: return fft_z_r2c_pipe_kernel<5>;
    case 6: return fft_z_r2c_pipe_kernel<6>;
    case 7: return fft_z_r2c_pipe_kernel<7>;
    case 8: return fft_z_r2c_pipe_kernel<8>;
    case 9: return fft_z_r2c_pipe_kernel<9>;
  }
  return nullptr;
}
ZC2RPipeFn z_c2r_pipe_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_c2r_pipe_kernel<3>;
    case 4: return fft_z_c2r_pipe_kernel<4>;
    case 5: return fft_z_c2r_pipe_kernel<5>;
    case 6: return fft_z_c2r_pipe_kernel<6>;
    case 7: return fft_z_c2r_pipe_kernel<7>;
    case 8: return fft_z_c2r_pipe_kernel<8>;
    case 9: return fft_z_c2r_pipe_kernel<9>;
  }
  return nullptr;
}

// shared memory of the persistent z passes: staging buffer + working tile
size_t z_pipe_smem(int lgM, bool c2r) {
  const int M = 1 << lgM, L = kZTile / M;
  const int stage = c2r ? ((L * (M + 1) + 1) & ~1) : L * M;
  return (size_t)(stage + L * zline_len(M)) * sizeof(float2);
}

int z_lines_per_cta(int Nz) { return kZTile / (Nz / 2); }

// the persistent z passes run when every array they copy in bulk starts 16-byte aligned and every
// tile's copy starts and ends on a 16-byte boundary: a complex line holds Nz/2 + 1 elements of 8
// bytes, an odd multiple of 8 bytes, so the lines per tile and the total line count must be even
// (an odd tile of C2R input would start 8 bytes off the boundary: a misaligned bulk copy)
template <class P>
bool z_pipe_ok(const pic_ctx* ctx, P const* p, int ncomp) {
  if (!ctx->dev_err || ctx->nsm <= 0 || (ctx->N[0] * ctx->N[1]) % 2 != 0) return false;
  if (z_lines_per_cta((int)ctx->N[2]) % 2 != 0) return false;
  for (int c = 0; c < ncomp; ++c)
    if (reinterpret_cast<uintptr_t>(p[c]) % 16 != 0) return false;
  return true;
}

template <class C> const C* twiddles(const pic_ctx* ctx, int a);
template <> const double2* twiddles<double2>(const pic_ctx* ctx, int a) { return ctx->twid[a]; }
template <> const float2* twiddles<float2>(const pic_ctx* ctx, int a) { return ctx->twid32[a]; }
template <class C> const C* pass_twiddles(const pic_ctx* ctx);
template <> const double2* pass_twiddles<double2>(const pic_ctx* ctx) { return ctx->twp; }
template <> const float2* pass_twiddles<float2>(const pic_ctx* ctx) { return ctx->twp32; }

template <class C>
pic_status launch_strided(pic_ctx* ctx, CP6<C> d, int axis, bool inv, int ncomp) {
  const int N = (int)ctx->N[axis];
  const int lgN = __builtin_ctz((unsigned)N);
  const int W = 1 << strided_lgw(lgN);
  const int nzh = (int)ctx->nzh;
  int64_t es, os, nouter;
  if (axis == 1) {  // y: outer = x
    es = nzh;
    os = ctx->N[1] * nzh;
    nouter = ctx->N[0];
  } else {  // x: outer = y
    es = ctx->N[1] * nzh;
    os = nzh;
    nouter = ctx->N[1];
  }
  StridedFn<C> fn = inv ? strided_fn<true, C>(lgN) : strided_fn<false, C>(lgN);
  if (!fn) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", N);
  dim3 grid((nzh + W - 1) / W, (unsigned)nouter, ncomp);
  const size_t smem = N > 8 ? (size_t)W * N * sizeof(C) : 0;
  fn<<<grid, W * N / 8, smem, ctx->stream>>>(d, es, os, nzh, pass_twiddles<C>(ctx));
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}


template <class T>
pic_status set_smem_attrs(pic_ctx* ctx) {
  using C = typename Cplx<T>::type;
  for (int lgM = 3; lgM <= 9; ++lgM) {
    const int zsm = (kZTile >> lgM) * zline_len(1 << lgM) * (int)sizeof(C);
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_r2c_fn<T>(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_c2r_fn<T>(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  }
  if (sizeof(T) == 4) {
    for (int lgM = 3; lgM <= 9; ++lgM) {
      PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_r2c_pipe_fn(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)z_pipe_smem(lgM, false)));
      PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_c2r_pipe_fn(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)z_pipe_smem(lgM, true)));
    }
  }
  for (int lgN = 4; lgN <= 10; ++lgN) {
    const int ssm = (1 << (lgN + strided_lgw(lgN))) * (int)sizeof(C);
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(strided_fn<false, C>(lgN), cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(strided_fn<true, C>(lgN), cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  }
  return PIC_OK;
}

}  // namespace

void sincospi_frac(int64_t p, int64_t q, double* s, double* c) {
  // sin, cos of pi p / q with the angle reduced on integers; exact at multiples of pi/2.
  int64_t r = p % (2 * q);
  if (r < 0) r += 2 * q;
  if ((2 * r) % q == 0) {
    const int64_t quarter = (2 * r) / q;  // 0..3
    const double sv[4] = {0.0, 1.0, 0.0, -1.0}, cv[4] = {1.0, 0.0, -1.0, 0.0};
    *s = sv[quarter];
    *c = cv[quarter];
    return;
  }
  const long double pi = 3.14159265358979323846264338327950288L;
  const long double a = pi * (long double)r / (long double)q;
  *s = (double)sinl(a);
  *c = (double)cosl(a);
}

pic_status fft_setup(pic_ctx* ctx) {
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      ctx->nsm = 0;
  }
  for (int a = 0; a < 3; ++a) {
    const int64_t N = ctx->N[a];
    double2* h = new double2[N];
    float2* hf = new float2[N];
    for (int64_t j = 0; j < N; ++j) {
      double s, c;
      sincospi_frac(2 * j, N, &s, &c);
      h[j] = make_double2(c, -s);  // exp(-2 pi i j / N)
      hf[j] = make_float2((float)c, (float)-s);
    }
    cudaError_t e = cudaMalloc(&ctx->twid[a], N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twid[a], h, N * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->twid32[a], N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twid32[a], hf, N * sizeof(float2), cudaMemcpyHostToDevice);
    delete[] h;
    delete[] hf;
    if (e != cudaSuccess) return pic_set_error(ctx, PIC_ERR_NOMEM, "twiddle table: %s", cudaGetErrorString(e));
  }
  {
    // per-pass tables (see pass_twiddle_offset): [r - 1][k] = exp(-2 pi i k r / (Ns R))
    double2* h = new double2[kPassTwiddles];
    float2* hf = new float2[kPassTwiddles];
    for (int lgNs = 3; lgNs <= 9; lgNs += 3) {
      for (int lgR = 3; lgR >= 1; --lgR) {
        const int Ns = 1 << lgNs, R = 1 << lgR, off = pass_twiddle_offset(lgNs, lgR);
        for (int r = 1; r < R; ++r)
          for (int k = 0; k < Ns; ++k) {
            double sn, cs;
            sincospi_frac(2 * (int64_t)k * r, (int64_t)Ns * R, &sn, &cs);
            h[off + (r - 1) * Ns + k] = make_double2(cs, -sn);
            hf[off + (r - 1) * Ns + k] = make_float2((float)cs, (float)-sn);
          }
      }
    }
    cudaError_t e = cudaMalloc(&ctx->twp, kPassTwiddles * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twp, h, kPassTwiddles * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->twp32, kPassTwiddles * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twp32, hf, kPassTwiddles * sizeof(float2), cudaMemcpyHostToDevice);
    delete[] h;
    delete[] hf;
    if (e != cudaSuccess) return pic_set_error(ctx, PIC_ERR_NOMEM, "twiddle table: %s", cudaGetErrorString(e));
  }
  pic_status st = set_smem_attrs<double>(ctx);
  if (st != PIC_OK) return st;
  return set_smem_attrs<float>(ctx);
}

template <class T>
pic_status fft_r2c(pic_ctx* ctx, CRP6<T> in, CP6<typename Cplx<T>::type> out, int ncomp) {
  using C = typename Cplx<T>::type;
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  const int lgM = __builtin_ctz((unsigned)(Nz / 2));
  if (lgM < 3 || lgM > 9) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", Nz);
  if constexpr (sizeof(T) == 4) {
    if (z_pipe_ok(ctx, in.p, ncomp)) {
      const int tpc = (int)((nlines + L - 1) / L);
      const ZPipe zp{nlines, tpc, tpc * ncomp, ctx->dev_err};
      const int grid = std::min(zp.ntiles, kZPipeCtasPerSm * ctx->nsm);
      z_r2c_pipe_fn(lgM)<<<grid, kZThreads, z_pipe_smem(lgM, false), ctx->stream>>>(in, out, zp,
                                                                                     twiddles<C>(ctx, 2),
                                                                                     pass_twiddles<C>(ctx));
      PIC_LAUNCH_CHECK(ctx);
      pic_status st = launch_strided<C>(ctx, out, 1, false, ncomp);
      if (st != PIC_OK) return st;
      return launch_strided<C>(ctx, out, 0, false, ncomp);
    }
  }
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  z_r2c_fn<T>(lgM)<<<grid, kZThreads, smem, ctx->stream>>>(in, out, nlines, twiddles<C>(ctx, 2),
                                                            pass_twiddles<C>(ctx));
  PIC_LAUNCH_CHECK(ctx);
  pic_status st = launch_strided<C>(ctx, out, 1, false, ncomp);
  if (st != PIC_OK) return st;
  return launch_strided<C>(ctx, out, 0, false, ncomp);
}

template <class T>
pic_status fft_c2r(pic_ctx* ctx, CP6<typename Cplx<T>::type> in, RP6<T> out, int ncomp) {
  using C = typename Cplx<T>::type;
  pic_status st = launch_strided<C>(ctx, in, 0, true, ncomp);
  if (st != PIC_OK) return st;
  st = launch_strided<C>(ctx, in, 1, true, ncomp);
  if (st != PIC_OK) return st;
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  const int lgM = __builtin_ctz((unsigned)(Nz / 2));
  if (lgM < 3 || lgM > 9) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", Nz);
  if constexpr (sizeof(T) == 4) {
    if (z_pipe_ok(ctx, in.p, ncomp)) {
      const int tpc = (int)((nlines + L - 1) / L);
      const ZPipe zp{nlines, tpc, tpc * ncomp, ctx->dev_err};
      const int grid = std::min(zp.ntiles, kZPipeCtasPerSm * ctx->nsm);
      z_c2r_pipe_fn(lgM)<<<grid, kZThreads, z_pipe_smem(lgM, true), ctx->stream>>>(in, out, zp,
                                                                                    twiddles<C>(ctx, 2),
                                                                                    pass_twiddles<C>(ctx));
      PIC_LAUNCH_CHECK(ctx);
      return PIC_OK;
    }
  }
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  z_c2r_fn<T>(lgM)<<<grid, kZThreads, smem, ctx->stream>>>(in, out, nlines, twiddles<C>(ctx, 2),
                                                            pass_twiddles<C>(ctx));
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

template pic_status fft_r2c<double>(pic_ctx*, CRP6<double>, CP6<double2>, int);
template pic_status fft_r2c<float>(pic_ctx*, CRP6<float>, CP6<float2>, int);
template pic_status fft_c2r<double>(pic_ctx*, CP6<double2>, RP6<double>, int);
template pic_status fft_c2r<float>(pic_ctx*, CP6<float2>, RP6<float>, int);
