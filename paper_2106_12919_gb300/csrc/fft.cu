// 3D real-to-complex FFT for the PSATD solver: shared-memory Stockham kernels,
// templated on the precision (FP64 form: double; FP32 form: float).
//
// Forward: z-axis R2C (a length-Nz/2 complex FFT of packed (even, odd) pairs
// followed by the split step), then in-place C2C along y and along x.
// Inverse: C2C along x, along y, then z-axis C2R.  Plain DFT, unnormalised:
// X_m = sum_j x_j exp(-2 pi i j.m / N) (App. A.1, Eq. Fourier_discrete without
// the half-cell phase, which the caller applies).
//
// Every CTA loads a whole tile of lines into shared memory, runs the radix-8
// (+ one radix-4 or radix-2) Stockham passes there, and writes the tile back.
// z lines are contiguous (line-major tile, padded one slot per 16 elements to
// spread the radix-8 scatter over the banks); y and x lines are strided, so a CTA
// takes W adjacent columns (consecutive k_z) and the tile is element-major,
// which keeps the global loads coalesced in W-element rows.
#include "pic_internal.cuh"
#include "fft_tile.cuh"

#include <cmath>

namespace {

constexpr int kZTile = 4096;    // complex elements per z-pass CTA (L lines * Nz/2)
constexpr int kMaxThreads = 1024;

using namespace pic_fft;

// z-axis real-to-complex: L lines of Nz reals -> Nz/2+1 complex per line.
template <class T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 3 : 2) fft_z_r2c_kernel(CRP6<T> in, CP6<typename Cplx<T>::type> out, int Nz,
                                                               int64_t nlines, int L,
                                                               const typename Cplx<T>::type* __restrict__ tw,
                                                               int bulk, int* err) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bar;
  C* sm = reinterpret_cast<C*>(smraw);
  const int M = Nz / 2;
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const C* src = reinterpret_cast<const C*>(in.p[comp]);
  if (bulk) {
    // the CTA's lines are contiguous in global memory: one bulk copy per 16-element segment into
    // its padded slot, issued by half of the threads, completing on one mbarrier
    const int lgM = lg2(M);
    const int lgS = lgM - kZPadShift;  // log2 segments per line
    const int nvalid = (int)min((int64_t)L, nlines - line0);
    const int nseg = nvalid << lgS;
    constexpr uint32_t seg_bytes = 16 * sizeof(C);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, (uint32_t)nseg * seg_bytes);
    for (int g = threadIdx.x; g < nseg; g += blockDim.x) {
      const int l = g >> lgS, k = g & ((1 << lgS) - 1);
      bulk_load(sm + lay.idx(k << kZPadShift, l), src + (line0 + l) * M + (k << kZPadShift), seg_bytes, &bar);
    }
    for (int t = (nvalid << lgM) + threadIdx.x; t < L * M; t += blockDim.x)  // lines past the end: zeros
      sm[lay.idx(t & (M - 1), t >> lgM)] = czero<C>();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      mbar_wait_bounded(&bar, 0);  // copies still in flight land before the CTA leaves
      return;
    }
  } else {
    // L * M == 8 * blockDim.x: 8 elements per thread, loads issued back to back
    C v[8];
    const int lgM = lg2(M);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int t = threadIdx.x + q * blockDim.x;
      const int l = t >> lgM;
      const int64_t line = line0 + l;
      v[q] = line < nlines ? src[line * M + (t & (M - 1))] : czero<C>();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int t = threadIdx.x + q * blockDim.x;
      sm[lay.idx(t & (M - 1), t >> lgM)] = v[q];
    }
  }
  __syncthreads();
  fft_tile<false>(sm, lay, M, tw, 2);
  // split: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W^k (Z_k - conj Z_{M-k}),  W = exp(-2 pi i / Nz)
  C* dst = out.p[comp];
  const int nzh = M + 1;
  const T h = (T)0.5;
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  const int lgH = lg2(M) - 1;
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
template <class T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 3 : 2) fft_z_c2r_kernel(CP6<typename Cplx<T>::type> in, RP6<T> out, int Nz,
                                                               int64_t nlines, int L,
                                                               const typename Cplx<T>::type* __restrict__ tw,
                                                               int bulk) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int M = Nz / 2;
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const C* srcb = in.p[comp];
  const int nzh = M + 1, P = M / 2 + 1;
  // Z_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  constexpr int kBatch = 5;  // L * P <= 5 * blockDim.x for every M >= 8 (L * M = 8 * blockDim.x)
  const int lgH = lg2(M) - 1;
  C xk[kBatch], xm[kBatch];
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
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
    const int t = threadIdx.x + q * blockDim.x;
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
  fft_tile<true>(sm, lay, M, tw, 2);
  C* dst = reinterpret_cast<C*>(out.p[comp]);
  const int lgM = lg2(M);
  if (bulk) {
    // one bulk copy per 16-element segment from its padded slot to the contiguous lines
    fence_proxy_async_shared();
    __syncthreads();
    const int lgS = lgM - kZPadShift;
    const int nvalid = (int)min((int64_t)L, nlines - line0);
    for (int g = threadIdx.x; g < (nvalid << lgS); g += blockDim.x) {
      const int l = g >> lgS, k = g & ((1 << lgS) - 1);
      bulk_store(dst + (line0 + l) * M + (k << kZPadShift), sm + lay.idx(k << kZPadShift, l), 16 * sizeof(C));
    }
    bulk_commit_and_wait_read();  // the shared memory is read before the CTA leaves
    return;
  }
  for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
    const int l = t >> lgM, e = t & (M - 1);
    const int64_t line = line0 + l;
    if (line < nlines) dst[line * M + e] = sm[lay.idx(e, l)];
  }
}

// In-place C2C along a strided axis: element e of column col of outer line o of
// component c at p[c] + o * os + e * es + col.  A CTA takes W adjacent columns.
// MAXT: the block size bound; the common 256-thread launches (N <= 128 with 16 columns) are
// compiled for 5 resident CTAs per SM in FP32 (48 registers, no spills) and 4 in FP64, larger ones
// for one.
template <bool INV, class C, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? (sizeof(C) == 8 ? 5 : 4) : 1) fft_strided_kernel(CP6<C> data, int N, int64_t es, int64_t os,
                                                                 int ncols, int W, const C* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int lgW = lg2(W);
  const LayCol lay{lgW};
  const int comp = blockIdx.z;
  const int col0 = blockIdx.x * W;
  C* base = data.p[comp] + (int64_t)blockIdx.y * os + col0;
  const int wv = min(W, ncols - col0);
  // N * W == 8 * blockDim.x: every thread moves 8 elements; the 8 loads are issued back to back
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    const int e = t >> lgW, w = t & (W - 1);
    v[q] = w < wv ? base[e * es + w] : czero<C>();
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) sm[threadIdx.x + q * blockDim.x] = v[q];
  __syncthreads();
  fft_tile<INV>(sm, lay, N, tw, 1);
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    const int e = t >> lgW, w = t & (W - 1);
    if (w < wv) base[e * es + w] = sm[t];
  }
}

// columns per CTA of the strided passes (measured: 16 and 8 equal, 32 slower)
int strided_width(int N) { return N >= 1024 ? 8 : 16; }

template <class C> const C* twiddles(const pic_ctx* ctx, int a);
template <> const double2* twiddles<double2>(const pic_ctx* ctx, int a) { return ctx->twid[a]; }
template <> const float2* twiddles<float2>(const pic_ctx* ctx, int a) { return ctx->twid32[a]; }

template <class C>
pic_status launch_strided(pic_ctx* ctx, CP6<C> d, int axis, bool inv, int ncomp) {
  const int N = (int)ctx->N[axis];
  const int W = strided_width(N);
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
  dim3 grid((nzh + W - 1) / W, (unsigned)nouter, ncomp);
  const int threads = W * N / 8;
  const size_t smem = (size_t)W * N * sizeof(C);
  const C* tw = twiddles<C>(ctx, axis);
  if (threads <= 256) {
    if (inv) fft_strided_kernel<true, C, 256><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, tw);
    else fft_strided_kernel<false, C, 256><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, tw);
  } else {
    if (inv) fft_strided_kernel<true, C, kMaxThreads><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, tw);
    else fft_strided_kernel<false, C, kMaxThreads><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, tw);
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

int z_lines_per_cta(int Nz) { return kZTile / (Nz / 2); }

// the z passes move lines by bulk copies when every real array starts 16-byte aligned and a line
// holds whole 16-element segments
template <class P>
bool bulk_ok(const pic_ctx* ctx, P const* p, int ncomp) {
  if (ctx->N[2] / 2 < 16 || !ctx->dev_err) return false;
  for (int c = 0; c < ncomp; ++c)
    if (reinterpret_cast<uintptr_t>(p[c]) % 16 != 0) return false;
  return true;
}

template <class T>
pic_status set_smem_attrs(pic_ctx* ctx) {
  using C = typename Cplx<T>::type;
  const int zsm = zline_len(kZTile) * (int)sizeof(C);
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_z_r2c_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_z_c2r_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  const int ssm = 8192 * (int)sizeof(C);
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<false, C, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<true, C, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<false, C, kMaxThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<true, C, kMaxThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
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
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  fft_z_r2c_kernel<T><<<grid, L * (Nz / 2) / 8, smem, ctx->stream>>>(in, out, Nz, nlines, L, twiddles<C>(ctx, 2),
                                                                      bulk_ok(ctx, in.p, ncomp) ? 1 : 0, ctx->dev_err);
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
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  fft_z_c2r_kernel<T><<<grid, L * (Nz / 2) / 8, smem, ctx->stream>>>(in, out, Nz, nlines, L, twiddles<C>(ctx, 2),
                                                                      bulk_ok(ctx, out.p, ncomp) ? 1 : 0);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

template pic_status fft_r2c<double>(pic_ctx*, CRP6<double>, CP6<double2>, int);
template pic_status fft_r2c<float>(pic_ctx*, CRP6<float>, CP6<float2>, int);
template pic_status fft_c2r<double>(pic_ctx*, CP6<double2>, RP6<double>, int);
template pic_status fft_c2r<float>(pic_ctx*, CP6<float2>, RP6<float>, int);
