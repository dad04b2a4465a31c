// Shared-memory Stockham FFT building blocks (radix 8, plus one radix-4 or radix-2 pass) of the
// transform kernels (fft.cu).  All sizes are powers of two: index arithmetic uses shifts and masks
// (lg* = log2).
#pragma once

#include "pic_internal.cuh"

namespace pic_fft {

// z-pass lines are padded one slot per 16 elements: the radix-8 scatter of pass 0 (outputs 8 j + r)
// then spreads a warp's lanes over all banks
constexpr int kZPadShift = 4;

// All sizes are powers of two: index arithmetic uses shifts and masks (lg* = log2).
__device__ __forceinline__ int lg2(int v) { return __ffs(v) - 1; }

struct LayLine {  // z pass: element e of line l at l * LP + e + e / 16, LP = M + M / 16
  int LP;
  __device__ __forceinline__ int idx(int e, int l) const { return l * LP + e + (e >> kZPadShift); }
  // butterfly b of nb = 2^lgnb per line -> line l, index j
  __device__ __forceinline__ void map(int b, int lgnb, int& l, int& j) const {
    l = b >> lgnb;
    j = b & ((1 << lgnb) - 1);
  }
};

struct LayCol {  // y / x pass: element e of column w at e * W + w, W = 2^lgW
  int lgW;
  __device__ __forceinline__ int idx(int e, int w) const { return (e << lgW) + w; }
  __device__ __forceinline__ void map(int b, int lgnb, int& l, int& j) const {
    j = b >> lgW;
    l = b & ((1 << lgW) - 1);
  }
};

// multiply by -i (forward) or +i (inverse)
template <bool INV, class C>
__device__ __forceinline__ C rot90(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <bool INV, class C>
__device__ __forceinline__ void dft4(C& y0, C& y1, C& y2, C& y3) {
  C t0 = cadd(y0, y2), t1 = csub(y0, y2);
  C t2 = cadd(y1, y3), t3 = rot90<INV>(csub(y1, y3));
  y0 = cadd(t0, t2);
  y2 = csub(t0, t2);
  y1 = cadd(t1, t3);
  y3 = csub(t1, t3);
}

template <int R, bool INV, class C>
__device__ __forceinline__ void dft(C* v) {
  using T = decltype(v[0].x);
  if (R == 2) {
    C a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {  // R == 8: radix-2 split over n and n+4, then two radix-4 DFTs
    const T r2 = (T)0.70710678118654752440;
    C b[4], c[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      b[n] = cadd(v[n], v[n + 4]);
      c[n] = csub(v[n], v[n + 4]);
    }
    // c_n *= w8^n, w8 = exp(-+ 2 pi i / 8)
    C c1 = c[1], c3 = c[3];
    if (INV) {
      c[1].x = (c1.x - c1.y) * r2; c[1].y = (c1.x + c1.y) * r2;
      c[3].x = (-c3.x - c3.y) * r2; c[3].y = (c3.x - c3.y) * r2;
    } else {
      c[1].x = (c1.x + c1.y) * r2; c[1].y = (c1.y - c1.x) * r2;
      c[3].x = (c3.y - c3.x) * r2; c[3].y = (-c3.x - c3.y) * r2;
    }
    c[2] = rot90<INV>(c[2]);
    dft4<INV>(b[0], b[1], b[2], b[3]);
    dft4<INV>(c[0], c[1], c[2], c[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = b[k];
      v[2 * k + 1] = c[k];
    }
  }
}

// Per-pass twiddle tables.  Pass (Ns, R) multiplies input r of butterfly k < Ns by
// w^{k r}, w = exp(-2 pi i / (Ns R)): a function of (Ns, R) only, not of the transform length.  One
// table holds every pass of every length up to 1024, r-major ([r - 1][k]), so the lanes of a warp,
// which hold consecutive k, read consecutive entries: one or two 128-byte lines per load, where
// the length-N table read at stride (N / (Ns R)) r spread a warp's loads over up to 28 lines.
// Sections for Ns = 8, 64, 512, each R = 8, 4, 2 (7, 3, 1 entries per k).
constexpr int kPassTwiddles = 6424;  // sum over Ns of 11 Ns
__host__ __device__ __forceinline__ constexpr int pass_twiddle_offset(int lgNs, int lgR) {
  return 11 * ((1 << lgNs) - 8) / 7 + (lgR == 3 ? 0 : (lgR == 2 ? 7 : 10)) * (1 << lgNs);
}

// One Stockham pass of radix R on all lines of the tile, in place.  The CTA has
// exactly L * N / 8 threads; each thread handles 8 / R butterflies.  twp: the per-pass tables.
template <int R, bool INV, class C, class LAY>
__device__ __forceinline__ void stockham_pass(C* s, const LAY& lay, int lgN, int lgNs, const C* __restrict__ twp) {
  constexpr int PER = 8 / R;
  constexpr int LGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  const int T = blockDim.x;
  const int lgnb = lgN - LGR;
  const int nb = 1 << lgnb, Ns = 1 << lgNs;
  C v[PER][R];
  int ol[PER], oj[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int b = threadIdx.x + q * T;
    int l, j;
    lay.map(b, lgnb, l, j);
    ol[q] = l;
    oj[q] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q][r] = s[lay.idx(j + r * nb, l)];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = oj[q], l = ol[q];
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      const C* t = twp + pass_twiddle_offset(lgNs, LGR) + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(&t[(r - 1) * Ns]);
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
    }
    dft<R, INV>(v[q]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[lay.idx(base + r * Ns, l)] = v[q][r];
  }
  __syncthreads();
}


// ---------------------------------------------------------------------------
// Transforms of a compile-time length N = 2^LGN: radix-8 passes p = 0, 1, ... (Ns = 8^p) and one
// radix-4 or radix-2 pass for the remaining bits; npass = ceil(LGN / 3).  Every index is a
// compile-time shift or mask, the first pass can take its inputs from registers (loaded straight
// from global memory) and the last pass can hand its outputs to global memory, so a transform moves
// through shared memory npass - 1 times.
// ---------------------------------------------------------------------------
template <int LGN>
struct Plan {
  static constexpr int npass = (LGN + 2) / 3;
};
// log2 of the radix of pass P
template <int LGN, int P>
struct PassLgR {
  static constexpr int value = LGN - 3 * P < 3 ? LGN - 3 * P : 3;
};

// passes P .. PEND - 1, shared memory to shared memory
template <bool INV, int LGN, int P, int PEND, class C, class LAY>
__device__ __forceinline__ void passes_ct(C* s, const LAY& lay, const C* __restrict__ twp) {
  if constexpr (P < PEND) {
    stockham_pass<1 << PassLgR<LGN, P>::value, INV>(s, lay, LGN, 3 * P, twp);
    passes_ct<INV, LGN, P + 1, PEND>(s, lay, twp);
  }
}

// pass 0 (radix 8, no twiddles) on this thread's butterfly (j, l): v[r] = element j + r N / 8 of
// line l; the outputs 8 j + r go to shared memory
template <bool INV, class C, class LAY>
__device__ __forceinline__ void pass0_from_regs(C* s, const LAY& lay, C (&v)[8], int j, int l) {
  dft<8, INV>(v);
#pragma unroll
  for (int r = 0; r < 8; ++r) s[lay.idx(8 * j + r, l)] = v[r];
  __syncthreads();
}

// the last pass (Ns = N / R), from shared memory; out(l, e, value) receives element e of line l
template <bool INV, int LGN, class C, class LAY, class OUT>
__device__ __forceinline__ void last_pass_to(const C* s, const LAY& lay, const C* __restrict__ twp, OUT&& out) {
  constexpr int P = Plan<LGN>::npass - 1;
  constexpr int LGR = PassLgR<LGN, P>::value;
  constexpr int R = 1 << LGR, PER = 8 / R;
  constexpr int lgnb = LGN - LGR, nb = 1 << lgnb;  // nb = Ns
  C v[PER][R];
  int ol[PER], oj[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    int l, j;
    lay.map(b, lgnb, l, j);
    ol[q] = l;
    oj[q] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q][r] = s[lay.idx(j + r * nb, l)];
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int k = oj[q];  // j < Ns: the butterfly's twiddle index and its first output
    if (P > 0) {
      const C* t = twp + pass_twiddle_offset(3 * P, LGR) + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(&t[(r - 1) * nb]);
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
    }
    dft<R, INV>(v[q]);
#pragma unroll
    for (int r = 0; r < R; ++r) out(ol[q], k + r * nb, v[q][r]);
  }
}

// padded length of a z-pass line of M elements
__host__ __device__ __forceinline__ int zline_len(int M) { return M + (M >> kZPadShift); }

// ---------------------------------------------------------------------------
// bulk copies (the TMA engine's cp.async.bulk) between global and shared memory, completed on an
// mbarrier; every wait is bounded and reports a timeout through a device flag
// ---------------------------------------------------------------------------
constexpr int kBulkWaitLimit = 1 << 22;  // try_wait polls before a wait gives up (far beyond any copy)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// wait for phase `phase` of the barrier, at most kBulkWaitLimit polls; false when it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (int it = 0; it < kBulkWaitLimit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// global -> shared, `bytes` (a multiple of 16, both addresses 16-byte aligned), completing on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// shared -> global, tracked by the issuing thread's bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// make this thread's shared-memory writes visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace pic_fft
