// Learned inflow generator on the tensor cores (tcgen05, bfloat16 operands,
// FP32 accumulation in tensor memory), with its training and its rollout
// into the solver's prescribed-inflow planes.
//
// The paper closes (Sec. V) with the prospect of replacing grid-resolved
// inflow turbulence by a synthetic one; this generator is that component.
// Network (feature maps channels-last, [pixel][channel], pixels j * nz + k of
// a periodic ny x nz plane, samples stacked):
//   h_1     = conv(W_in, x) + b_in                    x: q_t, q_{t-1}, zeros
//   h_{l+1} = h_l + conv(W_l, phi(h_l)) + b_l          l = 1 .. L
//   delta   = conv(W_out, phi(h_{L+1})) + b_out        q_{t+1} = q_t + delta
// conv: periodic 3 x 3 cross-correlation, phi(s) = s (s > 0), s / 8 else.
// Trained on mean-square error of delta with Adam on FP32 master weights;
// every convolution operand (weights, activations, back-propagated
// gradients) is bfloat16, the residual streams of h and of the gradient FP32.
//
// Kernels:
//  * k_conv: implicit-GEMM convolution, one CTA per 128 pixels of one image
//    row (nz a multiple of 128) and all N output channels. Per K block (one
//    tap row dy, 32 input channels) the CTA stages the 130-pixel row segment
//    (the z halo included) and the three taps' weights with 16-byte cp.async
//    copies into K-major core-matrix tiles whose pixel dimension is linear in
//    16-byte rows, so the three z taps are three start addresses of one tile;
//    one thread issues 3 x 2 MMAs (M = 128, N, K = 16) per block into a
//    tensor-memory accumulator, three shared-memory stages in flight. The
//    epilogue (bias, residual, activation, or the activation derivative for
//    the backward pass) runs on tcgen05.ld rows, one pixel per thread.
//    Forward and input-gradient passes are the same kernel: the input
//    gradient is a convolution with the flipped, transposed weights.
//  * k_wgrad: weight gradients dW[tap][o][c] = sum_p G[p][o] X[p + tap][c],
//    K = pixels: MN-major operand tiles straight from the channels-last maps
//    (a pixel's channels are one core-matrix row), the three z taps again as
//    start-address shifts of the haloed tile, three accumulators (one per
//    tap) in tensor memory; CTAs split the pixels, their partials are summed
//    in a fixed order (deterministic training).
//  * small kernels: input assembly, loss and its gradient, bias gradients,
//    Adam, weight packing, rollout statistics and emission.
// Every mbarrier wait is bounded; on expiry the kernel sets the error flag,
// waits (bounded) for its own tensor-core work, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ibm.h"
#include "common.cuh"
#include "tcgen05.cuh"

namespace ibm {

namespace {

using bf16 = __nv_bfloat16;

constexpr int CV_THREADS = 128;
constexpr int CV_M = 128;                   // pixels per tile
constexpr int CV_AROWS = CV_M + 2;          // with the z halo
constexpr uint32_t CV_ALBO = 138 * 16;      // K-group strip of the A tile (= 32 mod 128: no bank conflicts)
constexpr int CV_STAGES = 3;

template <int N, int KC>
struct ConvCfg {
  static constexpr int KB = KC < 32 ? KC : 32;     // input channels per K block
  static constexpr int KG = KB / 8;                // 16-byte K groups per block
  static constexpr int CB = KC / KB;               // channel blocks
  static constexpr int NK = 3 * CB;                // K blocks: tap rows x channel blocks
  static constexpr uint32_t A_BYTES = KG * CV_ALBO;
  static constexpr uint32_t B_LBO = N * 16 + 32;   // K-group strip of one tap's weights
  static constexpr uint32_t B_TAP = KG * B_LBO;
  static constexpr uint32_t STAGE = ((A_BYTES + 3 * B_TAP + 127) / 128) * 128;
  static constexpr uint32_t SMEM = CV_STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = N < 32 ? 32 : N;
};

__device__ inline float phi(float s) { return s > 0.f ? s : 0.125f * s; }

struct ConvArgs {
  const bf16* in;      // [pixels][KC]
  const bf16* w;       // [9 taps][N][KC]
  int ny, nz, rows;    // rows = samples * ny
  // epilogue: val = acc * (dact ? phi'(dact) : 1) + bias + res
  const bf16* dact;    // [pixels][N] or null
  const float* bias;   // [nbias] or null
  int nbias;
  const float* res;    // [pixels][N] or null
  float* out32;        // [pixels][ld32], channels < n32 (null: none)
  int ld32, n32;
  bf16* out16;         // [pixels][N] (null: none)
  int out16_phi;       // out16 = phi(val) instead of val
  int* error;
};

template <int N, int KC>
__global__ void __launch_bounds__(CV_THREADS, 2) k_conv(ConvArgs g) {
  using C = ConvCfg<N, KC>;
  extern __shared__ __align__(1024) unsigned char csm[];
  __shared__ uint64_t done[CV_STAGES];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_per_row = g.nz / CV_M;
  const int row = blockIdx.x / tiles_per_row;            // sample * ny + y
  const int z0 = (blockIdx.x - row * tiles_per_row) * CV_M;
  const int b = row / g.ny, y = row - b * g.ny;
  const uint32_t sbase = smem_u32(csm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < CV_STAGES; ++s) mbar_init(&done[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  auto load = [&](int kb, int s) {
    const int dyi = kb / C::CB, cb = kb - dyi * C::CB;
    int yy = y + dyi - 1;
    yy += (yy < 0) ? g.ny : 0;
    yy -= (yy >= g.ny) ? g.ny : 0;
    const size_t rbase = (size_t)(b * g.ny + yy) * g.nz;
    const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
    for (int e = tid; e < CV_AROWS * C::KG; e += CV_THREADS) {
      const int r = e / C::KG, kg = e - r * C::KG;
      int z = z0 - 1 + r;
      z += (z < 0) ? g.nz : 0;
      z -= (z >= g.nz) ? g.nz : 0;
      cp_async16(sa + (uint32_t)kg * CV_ALBO + (uint32_t)r * 16,
                 g.in + (rbase + z) * KC + cb * C::KB + kg * 8);
    }
    const uint32_t sb = sa + C::A_BYTES;
    for (int e = tid; e < 3 * N * C::KG; e += CV_THREADS) {
      const int kg = e % C::KG, n = (e / C::KG) % N, t = e / (C::KG * N);
      cp_async16(sb + (uint32_t)t * C::B_TAP + (uint32_t)kg * C::B_LBO + (uint32_t)n * 16,
                 g.w + ((size_t)((dyi * 3 + t) * N + n)) * KC + cb * C::KB + kg * 8);
    }
  };
  constexpr uint32_t idesc = tc_idesc_bf16(CV_M, N, false, false);
  auto issue = [&](int kb, int s) {
    const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
    const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int kk = 0; kk < C::KB / 16; ++kk) {
        const uint64_t ad = tc_desc(sa + (uint32_t)t * 16 + (uint32_t)kk * 2 * CV_ALBO, CV_ALBO, 128);
        const uint64_t bd = tc_desc(sb + (uint32_t)t * C::B_TAP + (uint32_t)kk * 2 * C::B_LBO, C::B_LBO, 128);
        tc_mma_bf16(tmem, ad, bd, idesc, (kb == 0 && t == 0 && kk == 0) ? 0u : 1u);
      }
    tc_commit_to(&done[s]);
  };

  bool ok = true;
#pragma unroll
  for (int i = 0; i < CV_STAGES - 1; ++i) {
    if (i < C::NK) load(i, i);
    cp_async_commit();
  }
  for (int kb = 0; kb < C::NK; ++kb) {
    const int s = kb % CV_STAGES;
    const int kn = kb + CV_STAGES - 1;
    if (kn < C::NK) {
      const int sn = kn % CV_STAGES;
      // the stage's previous MMAs (block kn - STAGES) must be done before it is overwritten
      if (kn >= CV_STAGES) ok = mbar_wait(&done[sn], (uint32_t)((kn - CV_STAGES) / CV_STAGES) & 1u) && ok;
      load(kn, sn);
    }
    cp_async_commit();
    cp_async_wait<CV_STAGES - 1>();   // this thread's copies of block kb have landed
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue(kb, s);
    }
  }
  ok = mbar_wait(&done[(C::NK - 1) % CV_STAGES], (uint32_t)((C::NK - 1) / CV_STAGES) & 1u) && ok;
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  if (ok) {
    const size_t p = (size_t)row * g.nz + z0 + warp * 32 + lane;
    constexpr int CW = N < 32 ? N : 32;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += CW) {
      float v[CW];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      if constexpr (CW == 32) tc_ld_x32(ta, v); else tc_ld_x16(ta, v);
      if (g.dact) {
        const bf16* da = g.dact + p * N + c0;
#pragma unroll
        for (int q = 0; q < CW; q += 8) {
          const uint4 raw = *reinterpret_cast<const uint4*>(da + q);
          const bf16* e = reinterpret_cast<const bf16*>(&raw);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[q + j] *= (__bfloat162float(e[j]) > 0.f) ? 1.f : 0.125f;
        }
      }
      if (g.bias) {
#pragma unroll
        for (int q = 0; q < CW; ++q) v[q] += (c0 + q < g.nbias) ? g.bias[c0 + q] : 0.f;
      }
      if (g.res) {
        const float* rr = g.res + p * N + c0;
#pragma unroll
        for (int q = 0; q < CW; q += 4) {
          const float4 t = *reinterpret_cast<const float4*>(rr + q);
          v[q] += t.x; v[q + 1] += t.y; v[q + 2] += t.z; v[q + 3] += t.w;
        }
      }
      if (g.out32) {
        float* o = g.out32 + p * g.ld32 + c0;
        if (g.ld32 == N) {
#pragma unroll
          for (int q = 0; q < CW; q += 4)
            *reinterpret_cast<float4*>(o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < CW; ++q)
            if (c0 + q < g.n32) o[q] = v[q];
        }
      }
      if (g.out16) {
        bf16* o = g.out16 + p * N + c0;
#pragma unroll
        for (int q = 0; q < CW; q += 8) {
          uint4 raw;
          bf16* e = reinterpret_cast<bf16*>(&raw);
#pragma unroll
          for (int j = 0; j < 8; ++j) e[j] = __float2bfloat16_rn(g.out16_phi ? phi(v[q + j]) : v[q + j]);
          *reinterpret_cast<uint4*>(o + q) = raw;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, C::TMEM_COLS);
}

// ---- weight gradients
constexpr int WG_THREADS = 128;
constexpr int WG_KP = 64;                  // pixels per K block
constexpr uint32_t WG_SBO_H = 67 * 16;     // 8-channel strip, 66 haloed rows (odd x 16: no bank conflicts)
constexpr uint32_t WG_SBO_P = 65 * 16;     // 8-channel strip, 64 rows
constexpr int WG_STAGES = 4;

template <int NB>
struct WgCfg {
  static constexpr uint32_t STAGE = ((16 * WG_SBO_H + (NB / 8) * WG_SBO_H + 127) / 128) * 128;
  static constexpr uint32_t SMEM = WG_STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = (3 * NB <= 64) ? 64 : 512;
};

struct WgArgs {
  const bf16* a;      // [pixels][128]: the M operand
  const bf16* b;      // [pixels][NB]:  the N operand
  int shift_a;        // the tap shift p + tap applies to a (else to b)
  int ny, nz, rows;   // rows = samples * ny
  int chunks;         // CTAs per tap row (gridDim.x)
  float* part;        // [3 dy][chunks][3 dz][128][NB]
  int* error;
};

template <int NB>
__global__ void __launch_bounds__(WG_THREADS, 1) k_wgrad(WgArgs g) {
  using C = WgCfg<NB>;
  extern __shared__ __align__(1024) unsigned char wsm[];
  __shared__ uint64_t done[WG_STAGES];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int dyi = blockIdx.y, chunk = blockIdx.x;
  const int per_row = g.nz / WG_KP;
  const int total = g.rows * per_row;
  const int per = (total + g.chunks - 1) / g.chunks;
  const int kb0 = chunk * per;
  const int nkb = max(0, min(total, kb0 + per) - kb0);
  const uint32_t sbo_a = g.shift_a ? WG_SBO_H : WG_SBO_P;
  const uint32_t sbo_b = g.shift_a ? WG_SBO_P : WG_SBO_H;
  const uint32_t a_bytes = 16 * sbo_a;
  const uint32_t sbase = smem_u32(wsm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < WG_STAGES; ++s) mbar_init(&done[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // one operand of one K block: `ch` channels of `nrows` pixels starting at
  // z = zs (wrapped) of image row rr, into 8-channel strips of stride sbo
  auto stage_operand = [&](uint32_t dst, const bf16* src, int ch, int rr, int zs, int nrows, uint32_t sbo) {
    const int groups = ch / 8;
    const size_t rbase = (size_t)rr * g.nz;
    for (int e = tid; e < nrows * groups; e += WG_THREADS) {
      const int r = e / groups, kg = e - r * groups;
      int z = zs + r;
      z += (z < 0) ? g.nz : 0;
      z -= (z >= g.nz) ? g.nz : 0;
      cp_async16(dst + (uint32_t)kg * sbo + (uint32_t)r * 16, src + (rbase + z) * ch + kg * 8);
    }
  };
  auto load = [&](int i, int s) {
    const int kb = kb0 + i;
    const int rr = kb / per_row, zb = (kb - rr * per_row) * WG_KP;
    const int bb = rr / g.ny, y = rr - bb * g.ny;
    int ys = y + dyi - 1;
    ys += (ys < 0) ? g.ny : 0;
    ys -= (ys >= g.ny) ? g.ny : 0;
    const int rs = bb * g.ny + ys;
    const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
    const uint32_t sb = sa + a_bytes;
    if (g.shift_a) {
      stage_operand(sa, g.a, 128, rs, zb - 1, WG_KP + 2, sbo_a);
      stage_operand(sb, g.b, NB, rr, zb, WG_KP, sbo_b);
    } else {
      stage_operand(sa, g.a, 128, rr, zb, WG_KP, sbo_a);
      stage_operand(sb, g.b, NB, rs, zb - 1, WG_KP + 2, sbo_b);
    }
  };
  constexpr uint32_t idesc = tc_idesc_bf16(128, NB, true, true);
  auto issue = [&](int i, int s) {
    const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
    const uint32_t sb = sa + a_bytes;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const uint32_t ao = g.shift_a ? (uint32_t)t * 16 : 0u;
      const uint32_t bo = g.shift_a ? 0u : (uint32_t)t * 16;
#pragma unroll
      for (int kk = 0; kk < WG_KP / 16; ++kk) {
        const uint64_t ad = tc_desc(sa + ao + (uint32_t)kk * 256, 128, sbo_a);
        const uint64_t bd = tc_desc(sb + bo + (uint32_t)kk * 256, 128, sbo_b);
        tc_mma_bf16(tmem + (uint32_t)(t * NB), ad, bd, idesc, (i == 0 && kk == 0) ? 0u : 1u);
      }
    }
    tc_commit_to(&done[s]);
  };

  bool ok = true;
#pragma unroll
  for (int i = 0; i < WG_STAGES - 1; ++i) {
    if (i < nkb) load(i, i);
    cp_async_commit();
  }
  for (int i = 0; i < nkb; ++i) {
    const int s = i % WG_STAGES;
    const int in = i + WG_STAGES - 1;
    if (in < nkb) {
      const int sn = in % WG_STAGES;
      if (in >= WG_STAGES) ok = mbar_wait(&done[sn], (uint32_t)((in - WG_STAGES) / WG_STAGES) & 1u) && ok;
      load(in, sn);
    }
    cp_async_commit();
    cp_async_wait<WG_STAGES - 1>();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue(i, s);
    }
  }
  if (nkb > 0) ok = mbar_wait(&done[(nkb - 1) % WG_STAGES], (uint32_t)((nkb - 1) / WG_STAGES) & 1u) && ok;
  cp_async_wait<0>();
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  if (ok) {
    const int m = warp * 32 + lane;
    float* out = g.part + ((size_t)(dyi * g.chunks + chunk) * 3) * 128 * NB;
    constexpr int CW = NB < 32 ? NB : 32;
#pragma unroll 1
    for (int t = 0; t < 3; ++t)
#pragma unroll 1
      for (int c0 = 0; c0 < NB; c0 += CW) {
        float v[CW];
        if (nkb > 0) {
          const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * NB + c0);
          if constexpr (CW == 32) tc_ld_x32(ta, v); else tc_ld_x16(ta, v);
        } else {
#pragma unroll
          for (int q = 0; q < CW; ++q) v[q] = 0.f;
        }
        float* o = out + ((size_t)t * 128 + m) * NB + c0;
#pragma unroll
        for (int q = 0; q < CW; q += 4) *reinterpret_cast<float4*>(o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, C::TMEM_COLS);
}

// grad[off + (tap O + o) C + c] = sum over chunks of the partials, for the
// real channels; `trans`: partial rows are input channels c, columns o
__global__ void k_wgrad_reduce(const float* __restrict__ part, int chunks, int NB, int trans, int O, int Cc,
                               float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * O * Cc) return;
  const int tap = i / (O * Cc), o = (i / Cc) % O, c = i % Cc;
  const int dyi = tap / 3, t = tap % 3;
  const int m = trans ? c : o, n = trans ? o : c;
  float s = 0.f;
  for (int k = 0; k < chunks; ++k) s += part[(((size_t)(dyi * chunks + k) * 3 + t) * 128 + m) * NB + n];
  grad[i] = s;
}

// bias gradients: per block, per lane of a stride S (a multiple of C) partial sums
__global__ void k_colsum_part(const float* __restrict__ x, size_t n, int S, double* __restrict__ part) {
  const int k = threadIdx.x;
  if (k >= S) return;
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = (size_t)blockIdx.x * per, hi = min(n, lo + per);
  double s = 0.0;
  long long r = ((long long)k - (long long)(lo % S)) % S;   // first index >= lo with i % S == k
  if (r < 0) r += S;
  for (size_t i = lo + (size_t)r; i < hi; i += S) s += x[i];
  part[(size_t)blockIdx.x * S + k] = s;
}

__global__ void k_colsum_final(const double* __restrict__ part, int blocks, int S, int Cc, float* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= Cc) return;
  double s = 0.0;
  for (int bl = 0; bl < blocks; ++bl)
    for (int k = c; k < S; k += Cc) s += part[(size_t)bl * S + k];
  out[c] = (float)s;
}

struct TIdx {
  int t[64];
};

// network input and target from raw planes [n][3][P]: x = (q_t, q_{t-1}, 0),
// target = q_{t+1} - q_t, q = (plane - mean) / std
__global__ void k_input_planes(const float* __restrict__ planes, int P, TIdx idx, int B, float3 mean, float3 istd,
                               bf16* __restrict__ x, float* __restrict__ target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P, p = i - b * P;
  const int t = idx.t[b];
  const float mu[3] = {mean.x, mean.y, mean.z}, is[3] = {istd.x, istd.y, istd.z};
  float qt[3], qp[3], qn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    qt[c] = (planes[((size_t)t * 3 + c) * P + p] - mu[c]) * is[c];
    qp[c] = (planes[((size_t)(t - 1) * 3 + c) * P + p] - mu[c]) * is[c];
    qn[c] = (planes[((size_t)(t + 1) * 3 + c) * P + p] - mu[c]) * is[c];
  }
  uint4 r0, r1;
  bf16* e0 = reinterpret_cast<bf16*>(&r0);
  bf16* e1 = reinterpret_cast<bf16*>(&r1);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    e0[j] = __float2bfloat16_rn(0.f);
    e1[j] = __float2bfloat16_rn(0.f);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    e0[c] = __float2bfloat16_rn(qt[c]);
    e0[3 + c] = __float2bfloat16_rn(qp[c]);
    target[(size_t)i * 3 + c] = qn[c] - qt[c];
  }
  reinterpret_cast<uint4*>(x + (size_t)i * 16)[0] = r0;
  reinterpret_cast<uint4*>(x + (size_t)i * 16)[1] = r1;
}

// network input from normalised planes [B][P][3]
__global__ void k_input_q(const float* __restrict__ qt, const float* __restrict__ qp, int n, bf16* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 r0, r1;
  bf16* e0 = reinterpret_cast<bf16*>(&r0);
  bf16* e1 = reinterpret_cast<bf16*>(&r1);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    e0[j] = __float2bfloat16_rn(0.f);
    e1[j] = __float2bfloat16_rn(0.f);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    e0[c] = __float2bfloat16_rn(qt[(size_t)i * 3 + c]);
    e0[3 + c] = __float2bfloat16_rn(qp[(size_t)i * 3 + c]);
  }
  reinterpret_cast<uint4*>(x + (size_t)i * 16)[0] = r0;
  reinterpret_cast<uint4*>(x + (size_t)i * 16)[1] = r1;
}

// gradient of the mean-square loss in delta (bf16, 16 channels, and FP32),
// per-block sums of the squared error
constexpr int LOSS_THREADS = 256;
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(const float* __restrict__ delta, const float* __restrict__ target,
                                                       int n, float scale, bf16* __restrict__ gd16,
                                                       float* __restrict__ gd32, double* __restrict__ part) {
  __shared__ double red[LOSS_THREADS];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double se = 0.0;
  if (i < n) {
    uint4 r0, r1;
    bf16* e0 = reinterpret_cast<bf16*>(&r0);
    bf16* e1 = reinterpret_cast<bf16*>(&r1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      e0[j] = __float2bfloat16_rn(0.f);
      e1[j] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float err = delta[(size_t)i * 3 + c] - target[(size_t)i * 3 + c];
      se += (double)err * err;
      const float gg = scale * err;
      gd32[(size_t)i * 3 + c] = gg;
      e0[c] = __float2bfloat16_rn(gg);
    }
    reinterpret_cast<uint4*>(gd16 + (size_t)i * 16)[0] = r0;
    reinterpret_cast<uint4*>(gd16 + (size_t)i * 16)[1] = r1;
  }
  red[threadIdx.x] = se;
  __syncthreads();
  for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_double(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// Adam; ob1 = 1 - b1, ob2 = 1 - b2 and the bias corrections c1 = 1 / (1 - b1^t),
// c2 = 1 / (1 - b2^t) come from the host in double, rounded once (1.f - 0.9f
// would carry the rounding of 0.9f into every step)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float ob1, float b2, float ob2,
                       float eps, float c1, float c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gg = gr[i];
  const float mi = b1 * m[i] + ob1 * gg;
  const float vi = b2 * v[i] + ob2 * gg * gg;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// bf16 operand copies of one layer's weights: wf[tap][Op][Cp] (forward) and
// wb[8 - tap][Cp][Op] (input gradient), zero in the padding
__global__ void k_pack(const float* __restrict__ w, int O, int Cc, int Op, int Cp, bf16* __restrict__ wf,
                       bf16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * Op * Cp) return;
  const int tap = i / (Op * Cp), o = (i / Cp) % Op, c = i % Cp;
  const float val = (o < O && c < Cc) ? w[((size_t)tap * O + o) * Cc + c] : 0.f;
  const bf16 hv = __float2bfloat16_rn(val);
  wf[i] = hv;
  if (wb) wb[((size_t)(8 - tap) * Cp + c) * Op + o] = hv;
}

// rollout: per-block sums of q = q_t + delta (pass 0) or of (q - mean)^2 (pass 1)
constexpr int ROLL_THREADS = 256;
__global__ void __launch_bounds__(ROLL_THREADS) k_roll_sums(const float* __restrict__ qt, const float* __restrict__ delta,
                                                            int P, const double* __restrict__ mean,
                                                            double* __restrict__ part) {
  __shared__ double red[3][ROLL_THREADS];
  const size_t per = ((size_t)P + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * per, hi = min((size_t)P, lo + per);
  double s[3] = {0.0, 0.0, 0.0};
  for (size_t p = lo + threadIdx.x; p < hi; p += ROLL_THREADS)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double q = (double)(qt[p * 3 + c] + delta[p * 3 + c]);
      s[c] += mean ? (q - mean[c]) * (q - mean[c]) : q;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = ROLL_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// pass 0: mean[c] = sum / P; pass 1: scale[c] = rms_target[c] / rms
__global__ void k_roll_stats(const double* __restrict__ part, int blocks, int P, int pass, double3 rms_target,
                             double* __restrict__ mean, double* __restrict__ scale) {
  const int c = threadIdx.x;
  if (c >= 3) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += part[b * 3 + c];
  if (pass == 0) {
    mean[c] = s / P;
  } else {
    const double tgt[3] = {rms_target.x, rms_target.y, rms_target.z};
    const double rms = sqrt(s / P);
    scale[c] = rms > 0.0 ? tgt[c] / rms : 1.0;
  }
}

// q_next = (q_t + delta - mean) * scale -> history; planes = mean_data + std * q_next
template <class T>
__global__ void k_roll_emit(const float* __restrict__ qt, const float* __restrict__ delta, int P,
                            const double* __restrict__ mean, const double* __restrict__ scale, float3 dmean,
                            float3 dstd, float* __restrict__ qnext, T* __restrict__ u, T* __restrict__ v,
                            T* __restrict__ w) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float mu[3] = {dmean.x, dmean.y, dmean.z}, sd[3] = {dstd.x, dstd.y, dstd.z};
  T* outs[3] = {u, v, w};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float q = (float)(((double)(qt[(size_t)p * 3 + c] + delta[(size_t)p * 3 + c]) - mean[c]) * scale[c]);
    qnext[(size_t)p * 3 + c] = q;
    if (outs[c]) outs[c][p] = (T)(mu[c] + sd[c] * q);
  }
}

// raw planes [3][P] -> normalised [P][3]
__global__ void k_normalise(const float* __restrict__ plane, int P, float3 mean, float3 istd, float* __restrict__ q) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  q[(size_t)p * 3 + 0] = (plane[p] - mean.x) * istd.x;
  q[(size_t)p * 3 + 1] = (plane[P + p] - mean.y) * istd.y;
  q[(size_t)p * 3 + 2] = (plane[2 * P + p] - mean.z) * istd.z;
}

template <int N, int KC>
void set_conv_attr() {
  cudaFuncSetAttribute(k_conv<N, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ConvCfg<N, KC>::SMEM);
}
template <int NB>
void set_wgrad_attr() {
  cudaFuncSetAttribute(k_wgrad<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WgCfg<NB>::SMEM);
}

template <int N, int KC>
void launch_conv(const ConvArgs& a, int tiles, cudaStream_t s) {
  k_conv<N, KC><<<tiles, CV_THREADS, ConvCfg<N, KC>::SMEM, s>>>(a);
}

template <int NB>
void launch_wgrad(const WgArgs& a, cudaStream_t s) {
  k_wgrad<NB><<<dim3(a.chunks, 3), WG_THREADS, WgCfg<NB>::SMEM, s>>>(a);
}

constexpr int WIDTH = 128;     // channels of the residual stream
constexpr int CIN_PAD = 16;    // input channels as stored (q_t, q_{t-1}, zeros)
constexpr int COUT_PAD = 16;   // output channels as computed (3 used)
constexpr int WG_CHUNKS = 50;  // CTAs per tap row of the weight gradients (3 x 50 <= 152 SMs)
constexpr int SUM_BLOCKS = 152;

struct Layer {
  int O, C, Op, Cp;        // real and padded output / input channels
  size_t woff, boff;       // offsets of W, b in the flat parameter array
  bf16* wf = nullptr;      // [9][Op][Cp]
  bf16* wb = nullptr;      // [9][Cp][Op]
};

}  // namespace

}  // namespace ibm

struct ibm_gen {
  int ny = 0, nz = 0, blocks = 0, cin = 0, batch = 0;
  size_t P = 0;
  cudaStream_t stream = nullptr;
  double lr = 1e-3, b1 = 0.9, b2 = 0.999, eps = 1e-8;
  long long t = 0;
  size_t np = 0;
  std::vector<ibm::Layer> layers;   // in, blocks..., out
  float *w = nullptr, *gw = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wpack = nullptr;
  __nv_bfloat16* x = nullptr;       // [B P][16]
  __nv_bfloat16* act = nullptr;     // (L + 1) maps [B P][128]: phi(h_1) .. phi(h_{L+1})
  __nv_bfloat16* g16[2] = {nullptr, nullptr};
  __nv_bfloat16* gd16 = nullptr;    // [B P][16]
  float* h[2] = {nullptr, nullptr};
  float* g32[2] = {nullptr, nullptr};
  float *delta = nullptr, *target = nullptr, *gd32 = nullptr;
  float* part = nullptr;            // weight-gradient partials
  double* dpart = nullptr;          // bias / loss / rollout partials
  double* dscal = nullptr;          // loss, rollout mean[3], scale[3]
  float* hist[2] = {nullptr, nullptr};
  int cur = 0;                      // hist[cur] = q_t, hist[cur ^ 1] = q_{t-1}
  float3 dmean = {0.f, 0.f, 0.f}, dstd = {1.f, 1.f, 1.f};
  double3 rms = {1.0, 1.0, 1.0};
  int* error = nullptr;
  std::vector<void*> allocs;
};

namespace {

using ibm::bf16;

int cuda_status(cudaError_t e) { return e == cudaSuccess ? IBM_OK : IBM_ECUDA; }

template <class T>
bool dalloc(ibm_gen* g, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return false;
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

bf16* act_map(ibm_gen* g, int l) { return g->act + (size_t)l * g->batch * g->P * ibm::WIDTH; }

int check_error(ibm_gen* g) {
  int e = 0;
  if (cudaMemcpyAsync(&e, g->error, sizeof(int), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess) return IBM_ECUDA;
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return IBM_ECUDA;
  if (e & ibm::ERR_TIMEOUT) return IBM_ETIMEOUT;
  return cuda_status(cudaGetLastError());
}

void pack_weights(ibm_gen* g) {
  for (auto& L : g->layers) {
    const int n = 9 * L.Op * L.Cp;
    ibm::k_pack<<<(n + 255) / 256, 256, 0, g->stream>>>(g->w + L.woff, L.O, L.C, L.Op, L.Cp, L.wf, L.wb);
  }
}

// forward pass of B samples whose input x is in place; delta -> g->delta
void forward(ibm_gen* g, int B) {
  using namespace ibm;
  const int rows = B * g->ny;
  const int tiles = rows * (g->nz / CV_M);
  ConvArgs a{};
  a.ny = g->ny; a.nz = g->nz; a.rows = rows; a.error = g->error;
  // h_1 = conv(W_in, x) + b_in; act_0 = phi(h_1)
  a.in = g->x; a.w = g->layers[0].wf; a.bias = g->w + g->layers[0].boff; a.nbias = WIDTH;
  a.out32 = g->h[0]; a.ld32 = WIDTH; a.n32 = WIDTH; a.out16 = act_map(g, 0); a.out16_phi = 1;
  launch_conv<WIDTH, CIN_PAD>(a, tiles, g->stream);
  for (int l = 1; l <= g->blocks; ++l) {
    const Layer& L = g->layers[l];
    ConvArgs c = a;
    c.in = act_map(g, l - 1); c.w = L.wf; c.bias = g->w + L.boff;
    c.res = g->h[(l - 1) & 1]; c.out32 = g->h[l & 1]; c.out16 = act_map(g, l);
    launch_conv<WIDTH, WIDTH>(c, tiles, g->stream);
  }
  const Layer& Lo = g->layers.back();
  ConvArgs o{};
  o.ny = g->ny; o.nz = g->nz; o.rows = rows; o.error = g->error;
  o.in = act_map(g, g->blocks); o.w = Lo.wf; o.bias = g->w + Lo.boff; o.nbias = 3;
  o.out32 = g->delta; o.ld32 = 3; o.n32 = 3;
  launch_conv<COUT_PAD, WIDTH>(o, tiles, g->stream);
}

void wgrad(ibm_gen* g, const bf16* a, const bf16* b, int nb, int shift_a, int trans, const ibm::Layer& L, int rows) {
  using namespace ibm;
  WgArgs w{};
  w.a = a; w.b = b; w.shift_a = shift_a; w.ny = g->ny; w.nz = g->nz; w.rows = rows;
  w.chunks = WG_CHUNKS; w.part = g->part; w.error = g->error;
  if (nb == WIDTH) launch_wgrad<WIDTH>(w, g->stream); else launch_wgrad<16>(w, g->stream);
  const int n = 9 * L.O * L.C;
  k_wgrad_reduce<<<(n + 255) / 256, 256, 0, g->stream>>>(g->part, WG_CHUNKS, nb, trans, L.O, L.C, g->gw + L.woff);
}

void colsum(ibm_gen* g, const float* x, size_t pixels, int C, float* out) {
  const int S = (C == 3) ? 96 : C;
  ibm::k_colsum_part<<<ibm::SUM_BLOCKS, 128, 0, g->stream>>>(x, pixels * C, S, g->dpart);
  ibm::k_colsum_final<<<1, 128, 0, g->stream>>>(g->dpart, ibm::SUM_BLOCKS, S, C, out);
}

// loss gradients of B samples whose input x and target are in place
void backward(ibm_gen* g, int B) {
  using namespace ibm;
  const int rows = B * g->ny;
  const size_t n = (size_t)B * g->P;
  const int tiles = rows * (g->nz / CV_M);
  forward(g, B);
  const int lb = (int)((n + LOSS_THREADS - 1) / LOSS_THREADS);
  k_loss<<<lb, LOSS_THREADS, 0, g->stream>>>(g->delta, g->target, (int)n, (float)(2.0 / (3.0 * n)), g->gd16,
                                             g->gd32, g->dpart);
  k_sum_double<<<1, 32, 0, g->stream>>>(g->dpart, lb, g->dscal);
  const Layer& Lo = g->layers.back();
  // output layer: dW_out^T = sum act_L[p + tap] gd[p]; db_out; g_{L+1} = phi' * conv(Wb_out, gd)
  wgrad(g, act_map(g, g->blocks), g->gd16, 16, 1, 1, Lo, rows);
  colsum(g, g->gd32, n, 3, g->gw + Lo.boff);
  ConvArgs a{};
  a.ny = g->ny; a.nz = g->nz; a.rows = rows; a.error = g->error;
  a.in = g->gd16; a.w = Lo.wb; a.dact = act_map(g, g->blocks);
  a.out32 = g->g32[0]; a.ld32 = WIDTH; a.n32 = WIDTH; a.out16 = g->g16[0];
  launch_conv<WIDTH, COUT_PAD>(a, tiles, g->stream);
  int cur = 0;
  for (int l = g->blocks; l >= 1; --l) {
    const Layer& L = g->layers[l];
    // dW_l = sum g_{l+1}[p] act_{l-1}[p + tap]; db_l = sum g_{l+1}
    wgrad(g, g->g16[cur], act_map(g, l - 1), WIDTH, 0, 0, L, rows);
    colsum(g, g->g32[cur], n, WIDTH, g->gw + L.boff);
    // g_l = g_{l+1} + phi'(h_l) * conv(Wb_l, g_{l+1})
    ConvArgs c{};
    c.ny = g->ny; c.nz = g->nz; c.rows = rows; c.error = g->error;
    c.in = g->g16[cur]; c.w = L.wb; c.dact = act_map(g, l - 1); c.res = g->g32[cur];
    c.out32 = g->g32[cur ^ 1]; c.ld32 = WIDTH; c.n32 = WIDTH; c.out16 = g->g16[cur ^ 1];
    launch_conv<WIDTH, WIDTH>(c, tiles, g->stream);
    cur ^= 1;
  }
  const Layer& Li = g->layers[0];
  wgrad(g, g->g16[cur], g->x, 16, 0, 0, Li, rows);
  colsum(g, g->g32[cur], n, WIDTH, g->gw + Li.boff);
}

void adam(ibm_gen* g) {
  g->t += 1;
  const double c1 = 1.0 / (1.0 - std::pow(g->b1, (double)g->t));
  const double c2 = 1.0 / (1.0 - std::pow(g->b2, (double)g->t));
  ibm::k_adam<<<(unsigned)((g->np + 255) / 256), 256, 0, g->stream>>>(
      g->w, g->gw, g->m, g->v, g->np, (float)g->lr, (float)g->b1, (float)(1.0 - g->b1), (float)g->b2,
      (float)(1.0 - g->b2), (float)g->eps, (float)c1, (float)c2);
  pack_weights(g);
}

int read_loss(ibm_gen* g, size_t n, double* loss) {
  double s = 0.0;
  if (cudaMemcpyAsync(&s, g->dscal, sizeof(double), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  const int st = check_error(g);
  if (st != IBM_OK) return st;
  if (loss) *loss = s / (3.0 * (double)n);
  return IBM_OK;
}

bool ready_attr() {
  static bool done = false;
  if (!done) {
    ibm::set_conv_attr<ibm::WIDTH, ibm::CIN_PAD>();
    ibm::set_conv_attr<ibm::WIDTH, ibm::WIDTH>();
    ibm::set_conv_attr<ibm::COUT_PAD, ibm::WIDTH>();
    ibm::set_conv_attr<ibm::WIDTH, ibm::COUT_PAD>();
    ibm::set_wgrad_attr<ibm::WIDTH>();
    ibm::set_wgrad_attr<16>();
    done = true;
  }
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace

extern "C" {

int ibm_gen_create(const ibm_gen_config* cfg, ibm_gen** out) {
  using namespace ibm;
  if (!cfg || !out) return IBM_EINVAL;
  *out = nullptr;
  if (cfg->ny < 1 || cfg->nz < CV_M || cfg->nz % CV_M != 0 || cfg->width != WIDTH || cfg->blocks < 0 ||
      cfg->blocks > 64 || cfg->in_channels < 1 || cfg->in_channels > 6 || cfg->batch < 1 || cfg->batch > 64)
    return IBM_EINVAL;
  if ((size_t)cfg->ny * cfg->nz > (size_t)1 << 24) return IBM_EINVAL;
  ibm_gen* g = new (std::nothrow) ibm_gen();
  if (!g) return IBM_ENOMEM;
  g->ny = cfg->ny; g->nz = cfg->nz; g->blocks = cfg->blocks; g->cin = cfg->in_channels; g->batch = cfg->batch;
  g->P = (size_t)cfg->ny * cfg->nz;
  g->stream = static_cast<cudaStream_t>(cfg->stream);
  if (cfg->lr > 0) g->lr = cfg->lr;
  if (cfg->beta1 > 0) g->b1 = cfg->beta1;
  if (cfg->beta2 > 0) g->b2 = cfg->beta2;
  if (cfg->eps > 0) g->eps = cfg->eps;
  // layers and flat parameter offsets: W [3][3][O][C] then b [O]
  size_t off = 0;
  auto add = [&](int O, int C, int Op, int Cp) {
    Layer L;
    L.O = O; L.C = C; L.Op = Op; L.Cp = Cp;
    L.woff = off; off += (size_t)9 * O * C;
    L.boff = off; off += (size_t)O;
    g->layers.push_back(L);
  };
  add(WIDTH, g->cin, WIDTH, CIN_PAD);
  for (int l = 0; l < g->blocks; ++l) add(WIDTH, WIDTH, WIDTH, WIDTH);
  add(3, WIDTH, COUT_PAD, WIDTH);
  g->np = off;
  size_t npack = 0;
  for (auto& L : g->layers) npack += (size_t)2 * 9 * L.Op * L.Cp;
  const size_t BP = (size_t)g->batch * g->P;
  bool ok = ready_attr();
  ok = ok && dalloc(g, &g->w, g->np) && dalloc(g, &g->gw, g->np) && dalloc(g, &g->m, g->np) &&
       dalloc(g, &g->v, g->np) && dalloc(g, &g->wpack, npack) && dalloc(g, &g->x, BP * CIN_PAD) &&
       dalloc(g, &g->act, (size_t)(g->blocks + 1) * BP * WIDTH) && dalloc(g, &g->g16[0], BP * WIDTH) &&
       dalloc(g, &g->g16[1], BP * WIDTH) && dalloc(g, &g->gd16, BP * COUT_PAD) && dalloc(g, &g->h[0], BP * WIDTH) &&
       dalloc(g, &g->h[1], BP * WIDTH) && dalloc(g, &g->g32[0], BP * WIDTH) && dalloc(g, &g->g32[1], BP * WIDTH) &&
       dalloc(g, &g->delta, BP * 3) && dalloc(g, &g->target, BP * 3) && dalloc(g, &g->gd32, BP * 3) &&
       dalloc(g, &g->part, (size_t)3 * WG_CHUNKS * 3 * 128 * WIDTH) &&
       dalloc(g, &g->dpart, (size_t)std::max<size_t>(SUM_BLOCKS * 128, BP / LOSS_THREADS + 1)) &&
       dalloc(g, &g->dscal, 8) && dalloc(g, &g->hist[0], g->P * 3) && dalloc(g, &g->hist[1], g->P * 3) &&
       dalloc(g, &g->error, 1);
  if (!ok) {
    ibm_gen_destroy(g);
    return IBM_ENOMEM;
  }
  bf16* pk = g->wpack;
  for (auto& L : g->layers) {
    L.wf = pk; pk += (size_t)9 * L.Op * L.Cp;
    L.wb = pk; pk += (size_t)9 * L.Op * L.Cp;
  }
  cudaMemsetAsync(g->w, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->gw, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->m, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->v, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->x, 0, BP * CIN_PAD * sizeof(bf16), g->stream);
  cudaMemsetAsync(g->hist[0], 0, g->P * 3 * sizeof(float), g->stream);
  cudaMemsetAsync(g->hist[1], 0, g->P * 3 * sizeof(float), g->stream);
  cudaMemsetAsync(g->error, 0, sizeof(int), g->stream);
  pack_weights(g);
  const int st = check_error(g);
  if (st != IBM_OK) {
    ibm_gen_destroy(g);
    return st;
  }
  *out = g;
  return IBM_OK;
}

size_t ibm_gen_param_count(const ibm_gen* g) { return g ? g->np : 0; }

int ibm_gen_set_params(ibm_gen* g, const double* w, size_t n) {
  if (!g || !w || n != g->np) return IBM_EINVAL;
  std::vector<float> f(n);
  for (size_t i = 0; i < n; ++i) f[i] = (float)w[i];
  if (cudaMemcpyAsync(g->w, f.data(), n * sizeof(float), cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  cudaMemsetAsync(g->m, 0, n * sizeof(float), g->stream);
  cudaMemsetAsync(g->v, 0, n * sizeof(float), g->stream);
  g->t = 0;
  pack_weights(g);
  return check_error(g);
}

static int get_flat(ibm_gen* g, const float* src, double* out, size_t n) {
  if (!g || !out || n != g->np) return IBM_EINVAL;
  std::vector<float> f(n);
  if (cudaMemcpyAsync(f.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  const int st = check_error(g);
  if (st != IBM_OK) return st;
  for (size_t i = 0; i < n; ++i) out[i] = f[i];
  return IBM_OK;
}

int ibm_gen_get_params(ibm_gen* g, double* w, size_t n) { return g ? get_flat(g, g->w, w, n) : IBM_EINVAL; }
int ibm_gen_get_grads(ibm_gen* g, double* d, size_t n) { return g ? get_flat(g, g->gw, d, n) : IBM_EINVAL; }

int ibm_gen_set_norm(ibm_gen* g, const double* mean, const double* std, const double* rms) {
  if (!g || !mean || !std || !rms) return IBM_EINVAL;
  for (int c = 0; c < 3; ++c)
    if (!(std[c] > 0.0) || !(rms[c] >= 0.0) || !std::isfinite(mean[c])) return IBM_EINVAL;
  g->dmean = make_float3((float)mean[0], (float)mean[1], (float)mean[2]);
  g->dstd = make_float3((float)std[0], (float)std[1], (float)std[2]);
  g->rms = make_double3(rms[0], rms[1], rms[2]);
  return IBM_OK;
}

int ibm_gen_forward(ibm_gen* g, const float* q_t, const float* q_prev, float* delta, int batch) {
  if (!g || !q_t || !q_prev || !delta || batch < 1 || batch > g->batch) return IBM_EINVAL;
  const size_t n = (size_t)batch * g->P;
  ibm::k_input_q<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(q_t, q_prev, (int)n, g->x);
  forward(g, batch);
  if (cudaMemcpyAsync(delta, g->delta, n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  return check_error(g);
}

int ibm_gen_grad(ibm_gen* g, const float* q_t, const float* q_prev, const float* target, int batch,
                 double* loss) {
  if (!g || !q_t || !q_prev || !target || batch < 1 || batch > g->batch) return IBM_EINVAL;
  const size_t n = (size_t)batch * g->P;
  ibm::k_input_q<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(q_t, q_prev, (int)n, g->x);
  if (cudaMemcpyAsync(g->target, target, n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  backward(g, batch);
  return read_loss(g, n, loss);
}

int ibm_gen_adam_step(ibm_gen* g) {
  if (!g) return IBM_EINVAL;
  adam(g);
  return check_error(g);
}

int ibm_gen_train_step(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch, double* loss) {
  if (!g || !planes || !t_idx || batch < 1 || batch > g->batch) return IBM_EINVAL;
  ibm::TIdx idx{};
  for (int b = 0; b < batch; ++b) {
    if (t_idx[b] < 1 || t_idx[b] + 1 >= n_planes) return IBM_EINVAL;
    idx.t[b] = t_idx[b];
  }
  const size_t n = (size_t)batch * g->P;
  const float3 istd = make_float3(1.f / g->dstd.x, 1.f / g->dstd.y, 1.f / g->dstd.z);
  ibm::k_input_planes<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(planes, (int)g->P, idx, batch, g->dmean,
                                                                          istd, g->x, g->target);
  backward(g, batch);
  adam(g);
  if (!loss) return cuda_status(cudaGetLastError());
  return read_loss(g, n, loss);
}

int ibm_gen_rollout_init(ibm_gen* g, const float* plane_prev, const float* plane_cur) {
  if (!g || !plane_prev || !plane_cur) return IBM_EINVAL;
  const float3 istd = make_float3(1.f / g->dstd.x, 1.f / g->dstd.y, 1.f / g->dstd.z);
  const unsigned nb = (unsigned)((g->P + 255) / 256);
  g->cur = 0;
  ibm::k_normalise<<<nb, 256, 0, g->stream>>>(plane_cur, (int)g->P, g->dmean, istd, g->hist[0]);
  ibm::k_normalise<<<nb, 256, 0, g->stream>>>(plane_prev, (int)g->P, g->dmean, istd, g->hist[1]);
  return check_error(g);
}

int ibm_gen_rollout(ibm_gen* g, void* u, void* v, void* w, int precision) {
  using namespace ibm;
  if (!g) return IBM_EINVAL;
  if (precision != IBM_FP64 && precision != IBM_FP32 && precision != IBM_MIXED) return IBM_EINVAL;
  const int P = (int)g->P;
  float* qt = g->hist[g->cur];
  float* qp = g->hist[g->cur ^ 1];
  k_input_q<<<(P + 255) / 256, 256, 0, g->stream>>>(qt, qp, P, g->x);
  forward(g, 1);
  const int nb = SUM_BLOCKS;
  double* mean = g->dscal + 1;
  double* scale = g->dscal + 4;
  k_roll_sums<<<nb, ROLL_THREADS, 0, g->stream>>>(qt, g->delta, P, nullptr, g->dpart);
  k_roll_stats<<<1, 32, 0, g->stream>>>(g->dpart, nb, P, 0, g->rms, mean, scale);
  k_roll_sums<<<nb, ROLL_THREADS, 0, g->stream>>>(qt, g->delta, P, mean, g->dpart);
  k_roll_stats<<<1, 32, 0, g->stream>>>(g->dpart, nb, P, 1, g->rms, mean, scale);
  // the new plane overwrites q_{t-1} (already consumed) and becomes q_t
  if (precision == IBM_FP64)
    k_roll_emit<double><<<(P + 255) / 256, 256, 0, g->stream>>>(qt, g->delta, P, mean, scale, g->dmean, g->dstd,
                                                                qp, (double*)u, (double*)v, (double*)w);
  else
    k_roll_emit<float><<<(P + 255) / 256, 256, 0, g->stream>>>(qt, g->delta, P, mean, scale, g->dmean, g->dstd,
                                                               qp, (float*)u, (float*)v, (float*)w);
  g->cur ^= 1;
  return cuda_status(cudaGetLastError());
}

int ibm_gen_history(ibm_gen* g, float* q_t, float* q_prev) {
  if (!g || !q_t || !q_prev) return IBM_EINVAL;
  const size_t bytes = g->P * 3 * sizeof(float);
  if (cudaMemcpyAsync(q_t, g->hist[g->cur], bytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
      cudaMemcpyAsync(q_prev, g->hist[g->cur ^ 1], bytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  return check_error(g);
}

int ibm_gen_sync(ibm_gen* g) { return g ? check_error(g) : IBM_EINVAL; }

void ibm_gen_destroy(ibm_gen* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (void* p : g->allocs) cudaFree(p);
  delete g;
}

}  // extern "C"
