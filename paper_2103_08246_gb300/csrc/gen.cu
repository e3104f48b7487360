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
//  * k_conv: implicit-GEMM convolution on tiles of 256 (or 128) pixels of
//    one image row (nz a multiple of 128) and all N output channels,
//    persistent (one CTA per SM) and warp-specialised. Feature maps are
//    bfloat16 in 16-byte granules of 8 channels, pixel-fastest within a
//    channel group, so per K block (one tap row dy, 32 input channels) one
//    thread fills a stage with bulk copies (cp.async.bulk): per 8-channel
//    group the haloed run of pixels into a K-major core-matrix strip whose
//    pixel dimension is linear in 16-byte rows (the three z taps and the two
//    128-pixel halves are then start addresses of one tile), and the three
//    taps' weights from a pre-packed image of the stage. One thread issues
//    3 x 2 x 2 MMAs (M = 128, N, K = 16) per block into the tile's two
//    tensor-memory accumulators. Four stages, hand-offs by mbarriers only.
//    Eight epilogue warps (bias, residual, activation, or the activation
//    derivative of the backward pass; tcgen05.ld rows, one pixel per
//    thread) drain one tile's accumulators while the MMAs fill the other
//    buffer. Forward and input-gradient passes are the same kernel: the
//    input gradient is a convolution with the flipped, transposed weights.
//  * k_wgrad: weight gradients dW[tap][o][c] = sum_p G[p][o] X[p + tap][c],
//    K = pixels: MN-major operand tiles bulk-copied from the granule maps
//    (8 channels of a pixel are one core-matrix row), the three z taps again
//    as start-address shifts of the haloed tile, three accumulators (one per
//    tap) in tensor memory; blocks of 128 pixels filled by bulk copies from
//    two threads (one per operand), three stages; CTAs split the pixels,
//    their partials are summed in a fixed order (deterministic training).
//  * small kernels: input assembly, loss and its gradient, bias gradients,
//    Adam, weight packing, rollout statistics and emission.
// Every mbarrier wait is bounded; on expiry the kernel sets the error flag,
// waits (bounded) for its own tensor-core work, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ibm.h"
#include "common.cuh"
#include "tcgen05.cuh"

namespace ibm {
// the FP32 2-D Hartley transform of 256 x 256 planes (poisson.cu)
bool dht2d_planes_fp32(const float* in, float* out, int nplanes, const float* tw, cudaStream_t s);
void poisson_set_attributes();
}  // namespace ibm

namespace ibm {

namespace {

using bf16 = __nv_bfloat16;

constexpr int CV_THREADS = 384;                // copy warp, MMA warp, 2 idle, 8 epilogue warps
constexpr int CV_EPI_THREADS = 256;
constexpr int CV_STAGES = 4;

template <int N, int KC, int TM>
struct ConvCfg {
  static constexpr int KB = KC < 32 ? KC : 32;     // input channels per K block
  static constexpr int KG = KB / 8;                // 16-byte K groups per block
  static constexpr int CB = KC / KB;               // channel blocks
  static constexpr int NK = 3 * CB;                // K blocks: tap rows x channel blocks
  static constexpr int AROWS = TM + 2;             // pixels with the z halo
  // K-group strip of the A tile: the haloed rows, rounded to = 32 mod 128 bytes
  // (the 8 threads of a shared-store phase then hit 8 distinct bank groups)
  static constexpr uint32_t ALBO = ((AROWS * 16 + 127 - 32) / 128) * 128 + 32;
  static constexpr uint32_t A_BYTES = KG * ALBO;
  static constexpr uint32_t B_LBO = N * 16 + 32;   // K-group strip of one tap's weights
  static constexpr uint32_t B_TAP = KG * B_LBO;
  static constexpr uint32_t STAGE = ((A_BYTES + 3 * B_TAP + 127) / 128) * 128;
  // a CTA holding all 512 tensor-memory columns asks for enough shared
  // memory that no second CTA fits on its SM
  static constexpr uint32_t SMEM =
      (2 * (TM / 128) * N >= 512 && CV_STAGES * STAGE < 120 * 1024) ? 120 * 1024 : CV_STAGES * STAGE;
};

__device__ inline float phi(float s) { return s > 0.f ? s : 0.125f * s; }

// bfloat16 maps are stored in 16-byte granules of 8 channels, pixel-fastest
// within a channel group, with one periodic halo granule at each end of every
// (row, group) run: slot z + 1 holds pixel z, slot 0 pixel nz - 1, slot
// nz + 1 pixel 0. A channel group of a haloed run of pixels is then one
// contiguous block (one bulk copy, one tensor-map box, no wrap).
__host__ __device__ inline size_t granule(size_t row, int group, int z, int C, int nz) {
  return (row * (size_t)(C / 8) + group) * (size_t)(nz + 2) + (size_t)(z + 1);
}
__host__ __device__ inline size_t map_elems(size_t rows, int C, int nz) { return rows * (size_t)(C / 8) * (nz + 2) * 8; }

// FP32 streams (the residual h and the back-propagated gradient, N = 128
// channels) in float4 granules, pixel-fastest within a 4-channel group:
// granule (row, group, z) at (row N/4 + group) nz + z, so that the epilogue's
// lanes (consecutive pixels) touch consecutive 16-byte granules
__host__ __device__ inline size_t f32_granule(size_t row, int group, int z, int N, int nz) {
  return (row * (size_t)(N / 4) + group) * (size_t)nz + (size_t)z;
}

// store granule (row, group, z) and its halo copy
__device__ inline void store_granule(bf16* map, size_t row, int group, int z, int C, int nz, uint4 v) {
  *reinterpret_cast<uint4*>(map + granule(row, group, z, C, nz) * 8) = v;
  if (z == 0) *reinterpret_cast<uint4*>(map + granule(row, group, nz, C, nz) * 8) = v;
  if (z == nz - 1) *reinterpret_cast<uint4*>(map + granule(row, group, -1, C, nz) * 8) = v;
}

// byte offset of weight (tap, row n, input channel k) in the shared-memory
// image of a convolution's B operand: per K block (tap row, channel block)
// the three taps' K-group strips of N rows x 16 bytes (+ 32 bytes of pad),
// exactly as a stage holds them, so that one bulk copy fills a stage
__host__ __device__ inline size_t wimg_off(int tap, int n, int k, int N, int KC) {
  const int KB = KC < 32 ? KC : 32, KG = KB / 8, CB = KC / KB;
  const size_t lbo = (size_t)N * 16 + 32;
  const int dyi = tap / 3, t = tap % 3, cb = k / KB, kg = (k % KB) / 8, e = k % 8;
  return ((((size_t)(dyi * CB + cb) * 3 + t) * KG + kg) * lbo) + (size_t)n * 16 + (size_t)e * 2;
}
__host__ __device__ inline size_t wimg_bytes(int N, int KC) { return (size_t)9 * (KC / 8) * ((size_t)N * 16 + 32); }

// 1-D bulk copy of `bytes` to a shared address, completing on `bar`
__device__ inline void bulk_g2s_u32(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst), "l"(src),
      "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// bulk copy of the tensor-map box at coordinates (x, y, z) of a 3-D map
__device__ inline void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct ConvArgs {
  const bf16* in;      // KC-channel map, granule layout
  const unsigned char* w;   // B-operand image (wimg_off)
  int ny, nz, rows;    // rows = samples * ny
  // epilogue: val = acc * (dact ? phi'(dact) : 1) + bias + res
  const bf16* dact;    // N-channel map (granule layout) or null
  const float* bias;   // [nbias] or null
  int nbias;
  const float* res;    // FP32 stream (f32_granule layout) or null
  float* out32;        // ld32 == N: FP32 stream (f32_granule layout); else [pixels][ld32], channels < n32
  int ld32, n32;
  bf16* out16;         // N-channel map, granule layout (null: none)
  int out16_phi;       // out16 = phi(val) instead of val
  int* error;
};

// epilogue of CW accumulator columns c0 .. c0 + CW - 1 of pixel p = (row, z)
// (16-byte accesses, the loads of a chunk issued before the arithmetic; the
// bfloat16 granules of consecutive lanes are consecutive)
template <int N, int CW>
__device__ inline void conv_epilogue(const ConvArgs& g, size_t row, int z, int c0, float (&v)[CW]) {
  const size_t p = row * g.nz + z;
  if (g.dact) {
    uint4 raw[CW / 8];
#pragma unroll
    for (int q = 0; q < CW / 8; ++q)
      raw[q] = *reinterpret_cast<const uint4*>(g.dact + granule(row, c0 / 8 + q, z, N, g.nz) * 8);
#pragma unroll
    for (int q = 0; q < CW / 8; ++q) {
      const bf16* e = reinterpret_cast<const bf16*>(&raw[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[8 * q + j] *= (__bfloat162float(e[j]) > 0.f) ? 1.f : 0.125f;
    }
  }
  if (g.bias) {
#pragma unroll
    for (int q = 0; q < CW; ++q) v[q] += (c0 + q < g.nbias) ? g.bias[c0 + q] : 0.f;
  }
  if (g.res) {
    float4 t[CW / 4];
    const float4* rr = reinterpret_cast<const float4*>(g.res);
#pragma unroll
    for (int q = 0; q < CW / 4; ++q) t[q] = rr[f32_granule(row, c0 / 4 + q, z, N, g.nz)];
#pragma unroll
    for (int q = 0; q < CW / 4; ++q) {
      v[4 * q] += t[q].x; v[4 * q + 1] += t[q].y; v[4 * q + 2] += t[q].z; v[4 * q + 3] += t[q].w;
    }
  }
  if (g.out32) {
    float* o = g.out32 + p * g.ld32 + c0;
    if (g.ld32 == N) {   // an FP32 stream: granule layout
      float4* o4 = reinterpret_cast<float4*>(g.out32);
#pragma unroll
      for (int q = 0; q < CW; q += 4)
        o4[f32_granule(row, (c0 + q) / 4, z, N, g.nz)] = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    } else {
#pragma unroll
      for (int q = 0; q < CW; ++q)
        if (c0 + q < g.n32) o[q] = v[q];
    }
  }
  if (g.out16) {
#pragma unroll
    for (int q = 0; q < CW / 8; ++q) {
      uint4 raw;
      bf16* e = reinterpret_cast<bf16*>(&raw);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float x = v[8 * q + j];
        e[j] = __float2bfloat16_rn(g.out16_phi ? phi(x) : x);
      }
      store_granule(g.out16, row, c0 / 8 + q, z, N, g.nz, raw);
    }
  }
}

// Persistent, warp-specialised: CTA c takes tiles c, c + gridDim.x, ... (a
// tile is TM consecutive pixels of one image row, all N output channels).
//  * warp 0 (one thread) copies: for each K block j of the CTA's tiles (one
//    sequence over its tiles) it waits for the stage to be free (the tensor
//    core's commit of block j - STAGES), announces the stage's bytes on its
//    `full` barrier and issues bulk copies: per K group the haloed run of
//    pixels (one to three copies), and the three taps' weights (one copy of
//    the pre-packed image);
//  * warp 1 (one thread) waits for `full`, issues the block's MMAs into the
//    tile's tensor-memory buffer (two buffers, alternating by tile) and
//    commits them to the stage's `empty` barrier, after the tile's last
//    block also to the buffer's `tfull` barrier;
//  * warps 4-11 run the epilogue of tile i from its buffer (two warps per
//    lane quarter, each half of the columns) while the MMAs of tile i + 1
//    fill the other one, then arrive on the buffer's `tempty`.
template <int N, int KC, int TM>
__global__ void __launch_bounds__(CV_THREADS, 1) k_conv(ConvArgs g) {
  using C = ConvCfg<N, KC, TM>;
  constexpr int BUF_COLS = (TM / 128) * N;                       // one tile's accumulators
  constexpr uint32_t COLS = 2 * BUF_COLS < 32 ? 32 : 2 * BUF_COLS;
  constexpr uint32_t A_TX = (uint32_t)C::KG * C::AROWS * 16;
  constexpr uint32_t B_TX = 3 * C::B_TAP;
  extern __shared__ __align__(1024) unsigned char csm[];
  __shared__ uint64_t full[CV_STAGES], empty[CV_STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_per_row = g.nz / TM;
  const int ntiles = g.rows * tiles_per_row;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = my_tiles * C::NK;
  const uint32_t sbase = smem_u32(csm);

  if (warp == 0) tc_alloc(&tmem_slot, COLS);
  if (tid == 0) {
    for (int s = 0; s < CV_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], CV_EPI_THREADS);
    }
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      for (int j = 0; j < total; ++j) {
        const int s = j % CV_STAGES;
        if (j >= CV_STAGES) ok = mbar_wait(&empty[s], (uint32_t)((j - CV_STAGES) / CV_STAGES) & 1u) && ok;
        const int tile = blockIdx.x + (j / C::NK) * gridDim.x;
        const int kb = j % C::NK;
        const int row = tile / tiles_per_row, z0 = (tile - row * tiles_per_row) * TM;
        const int b = row / g.ny, y = row - b * g.ny;
        const int dyi = kb / C::CB, cb = kb - dyi * C::CB;
        int yy = y + dyi - 1;
        yy += (yy < 0) ? g.ny : 0;
        yy -= (yy >= g.ny) ? g.ny : 0;
        const size_t rr = (size_t)(b * g.ny + yy);
        const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
        mbar_arrive_expect_tx(&full[s], A_TX + B_TX);
        const char* src = reinterpret_cast<const char*>(g.in) + granule(rr, cb * C::KG, z0 - 1, KC, g.nz) * 16;
        if (C::ALBO == (uint32_t)(g.nz + 2) * 16) {   // the groups' runs are adjacent here too: one copy
          bulk_g2s_u32(sa, src, A_TX, &full[s]);
        } else {
#pragma unroll
          for (int kg = 0; kg < C::KG; ++kg)
            bulk_g2s_u32(sa + (uint32_t)kg * C::ALBO, src + (size_t)kg * (g.nz + 2) * 16, C::AROWS * 16, &full[s]);
        }
        bulk_g2s_u32(sa + C::A_BYTES, g.w + (size_t)(dyi * C::CB + cb) * B_TX, B_TX, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc_bf16(128, N, false, false);
      for (int j = 0; j < total; ++j) {
        const int s = j % CV_STAGES;
        const int lt = j / C::NK, kb = j % C::NK;
        // the buffer's previous tile (lt - 2) must have been read out
        if (kb == 0 && lt >= 2) ok = mbar_wait(&tempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        ok = mbar_wait(&full[s], (uint32_t)(j / CV_STAGES) & 1u) && ok;
        tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)((lt & 1) * BUF_COLS);
        const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
        const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
        for (int t = 0; t < 3; ++t)
#pragma unroll
          for (int kk = 0; kk < C::KB / 16; ++kk) {
            const uint64_t bd =
                tc_desc(sb + (uint32_t)t * C::B_TAP + (uint32_t)kk * 2 * C::B_LBO, C::B_LBO, 128);
#pragma unroll
            for (int h = 0; h < TM / 128; ++h) {   // 128-pixel halves: rows h * 128 .. of the tile
              const uint64_t ad =
                  tc_desc(sa + (uint32_t)(t + h * 128) * 16 + (uint32_t)kk * 2 * C::ALBO, C::ALBO, 128);
              tc_mma_bf16(dbase + (uint32_t)(h * N), ad, bd, idesc, (kb == 0 && t == 0 && kk == 0) ? 0u : 1u);
            }
          }
        tc_commit_to(&empty[s]);
        if (kb == C::NK - 1) tc_commit_to(&tfull[lt & 1]);
      }
    }
  } else if (warp >= 4) {
    // epilogue warps 4 .. 11: lane quarter warp % 4; warps w and w + 4 split
    // the columns (narrow outputs: warps 4 .. 7 take all of them)
    const int quarter = warp & 3, part = (warp - 4) >> 2;
    constexpr int CW = N < 32 ? N : 32;
    constexpr int SPLIT = N >= 64 ? 2 : 1;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int tile = blockIdx.x + lt * gridDim.x;
      const int row = tile / tiles_per_row, z0 = (tile - row * tiles_per_row) * TM;
      ok = mbar_wait(&tfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      tc_fence_after();
      const uint32_t dbase = tmem + (uint32_t)((lt & 1) * BUF_COLS);
#pragma unroll 1
      for (int h = 0; h < TM / 128; ++h) {
        const int z = z0 + h * 128 + quarter * 32 + lane;
#pragma unroll 1
        for (int c0 = part * (N / SPLIT); c0 < (part + 1) * (N / SPLIT) && part < SPLIT; c0 += CW) {
          float v[CW];
          const uint32_t ta = dbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(h * N + c0);
          if constexpr (CW == 32) tc_ld_x32(ta, v); else tc_ld_x16(ta, v);
          conv_epilogue<N, CW>(g, (size_t)row, z, c0, v);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[lt & 1]);
    }
  }
  // every MMA has completed once the last tile's buffer was committed
  if (tid == 32 && my_tiles > 0)
    ok = mbar_wait(&tfull[(my_tiles - 1) & 1], (uint32_t)((my_tiles - 1) / 2) & 1u) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, COLS);
}

// ---- weight gradients
constexpr int WG_THREADS = 256;
constexpr int WG_KP = 128;                 // pixels per K block
constexpr uint32_t WG_SBO_H = (WG_KP + 2) * 16;   // 8-channel strip of the haloed operand (a box row block)
constexpr uint32_t WG_SBO_P = WG_KP * 16;         // 8-channel strip of the other operand
constexpr int WG_STAGES = 3;

template <int NB>
struct WgCfg {
  static constexpr uint32_t STAGE = ((16 * WG_SBO_H + (NB / 8) * WG_SBO_H + 127) / 128) * 128;
  static constexpr uint32_t SMEM = WG_STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = (3 * NB <= 64) ? 64 : 512;
};

struct WgArgs {
  const bf16* a;      // 128-channel map (granule layout): the M operand
  const bf16* b;      // NB-channel map (granule layout): the N operand
  int shift_a;        // the tap shift p + tap applies to a (else to b)
  int ny, nz, rows;   // rows = samples * ny
  int chunks;         // CTAs per tap row (gridDim.x)
  float* part;        // [3 dy][chunks][3 dz][128][NB]
  int* error;
};

// Two threads fill the stages, one tensor-map box per operand and stage
// (warp 0: the M operand, all 16 channel groups of the run of pixels; warp 2:
// the N operand; the shifted one with its halo, which the maps store), warp 1
// (one thread) issues the MMAs; after the last block all warps read the three
// accumulators out. Maps: 3-D (8 channels, nz + 2 slots, rows x groups),
// boxes (8, 128 or 130, groups): the box lands as [group][pixel][8], the
// MN-major core-matrix strips.
template <int NB>
__global__ void __launch_bounds__(WG_THREADS, 1) k_wgrad(WgArgs g, const __grid_constant__ CUtensorMap map_a,
                                                        const __grid_constant__ CUtensorMap map_b) {
  using C = WgCfg<NB>;
  extern __shared__ __align__(1024) unsigned char wsm[];
  __shared__ uint64_t full[WG_STAGES], empty[WG_STAGES];
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
  const uint32_t rows_a = g.shift_a ? WG_KP + 2 : WG_KP, rows_b = g.shift_a ? WG_KP : WG_KP + 2;
  const uint32_t sbase = smem_u32(wsm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < WG_STAGES; ++s) {
      mbar_init(&full[s], 2);
      mbar_init(&empty[s], 1);
    }
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if ((warp == 0 || warp == 2) && lane == 0) {
    const bool is_a = warp == 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % WG_STAGES;
      if (i >= WG_STAGES) ok = mbar_wait(&empty[s], (uint32_t)((i - WG_STAGES) / WG_STAGES) & 1u) && ok;
      const int kb = kb0 + i;
      const int rr = kb / per_row, zb = (kb - rr * per_row) * WG_KP;
      const int bb = rr / g.ny, y = rr - bb * g.ny;
      int ys = y + dyi - 1;
      ys += (ys < 0) ? g.ny : 0;
      ys -= (ys >= g.ny) ? g.ny : 0;
      const int rs = bb * g.ny + ys;
      const uint32_t sa = sbase + (uint32_t)s * C::STAGE;
      if (is_a) {
        mbar_arrive_expect_tx(&full[s], 16 * rows_a * 16);
        const int ra = g.shift_a ? rs : rr, za = g.shift_a ? zb - 1 : zb;
        tma_load_3d(sa, &map_a, 0, za + 1, ra * 16, &full[s]);
      } else {
        mbar_arrive_expect_tx(&full[s], (NB / 8) * rows_b * 16);
        const int rb = g.shift_a ? rr : rs, zbb = g.shift_a ? zb : zb - 1;
        tma_load_3d(sa + a_bytes, &map_b, 0, zbb + 1, rb * (NB / 8), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc_bf16(128, NB, true, true);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % WG_STAGES;
        ok = mbar_wait(&full[s], (uint32_t)(i / WG_STAGES) & 1u) && ok;
        tc_fence_after();
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
        tc_commit_to(&empty[s]);
      }
      if (nkb > 0) ok = mbar_wait(&empty[(nkb - 1) % WG_STAGES], (uint32_t)((nkb - 1) / WG_STAGES) & 1u) && ok;
    }
  }
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  if (ok) {
    const int quarter = warp & 3, part = warp >> 2;
    float* out = g.part + ((size_t)(dyi * g.chunks + chunk) * 3) * 128 * NB;
    float* tr = reinterpret_cast<float*>(wsm) + warp * 32 * 33;   // the stages are free now
    constexpr int CW = NB < 32 ? NB : 32;
    constexpr int SPLIT = NB >= 64 ? 2 : 1;
    if (part < SPLIT) {
#pragma unroll 1
      for (int t = 0; t < 3; ++t)
#pragma unroll 1
        for (int c0 = part * (NB / SPLIT); c0 < (part + 1) * (NB / SPLIT); c0 += CW) {
          float v[CW];
          if (nkb > 0) {
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * NB + c0);
            if constexpr (CW == 32) tc_ld_x32(ta, v); else tc_ld_x16(ta, v);
          } else {
#pragma unroll
            for (int q = 0; q < CW; ++q) v[q] = 0.f;
          }
          // transpose through the warp's tile: row j of the partial, lanes = columns
#pragma unroll
          for (int q = 0; q < CW; ++q) tr[lane * 33 + q] = v[q];
          __syncwarp();
          if (lane < CW)
#pragma unroll 4
            for (int j = 0; j < 32; ++j)
              out[((size_t)t * 128 + quarter * 32 + j) * NB + c0 + lane] = tr[j * 33 + lane];
          __syncwarp();
        }
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

// bias gradient of the 3-channel output: the flat array [pixels][3] is split
// into equal runs, one per block (a multiple of the block's span, blockDim, a
// multiple of 3); thread t sums the elements t, t + span, ... of its run
// (about a hundred values, in FP32: the FP64 pipe of this part is far too
// narrow for per-element double additions) into entry t of its block's
// partial row (channel t mod 3); the partials are added in FP64.
constexpr int COLSUM_BLOCKS = 608;   // 4 per SM
__global__ void __launch_bounds__(256) k_colsum_part(const float* __restrict__ x, size_t n, double* __restrict__ part) {
  const size_t per = ((n + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const size_t lo = (size_t)blockIdx.x * per, hi = min(n, lo + per);
  float s0 = 0.f, s1 = 0.f;
  const size_t st = blockDim.x;
  size_t i = lo + threadIdx.x;
  for (; i + st < hi; i += 2 * st) {
    s0 += x[i];
    s1 += x[i + st];
  }
  for (; i < hi; i += st) s0 += x[i];
  part[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s0 + (double)s1;
}

// bias gradients of an FP32 stream (f32_granule layout, N channels): one
// block per (row, 4-channel group) sums its run of nz granules (FP32 per
// thread), partial row per image row: part[row][N]
__global__ void __launch_bounds__(64) k_colsum_stream(const float4* __restrict__ x, int nz, int N,
                                                      double* __restrict__ part) {
  __shared__ float4 red[64];
  const size_t run = blockIdx.x;   // row * N/4 + group
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int z = threadIdx.x; z < nz; z += 64) {
    const float4 a = x[run * nz + z];
    s.x += a.x; s.y += a.y; s.z += a.z; s.w += a.w;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 32; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
      red[threadIdx.x].z += red[threadIdx.x + w].z;
      red[threadIdx.x].w += red[threadIdx.x + w].w;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* o = part + run * 4;   // = row * N + 4 group
    o[0] = red[0].x; o[1] = red[0].y; o[2] = red[0].z; o[3] = red[0].w;
  }
}

// one block per channel: the entries e = c mod C of every block's partial
// row (S entries), summed in a fixed order (deterministic)
__global__ void __launch_bounds__(256) k_colsum_final(const double* __restrict__ part, int blocks, int S, int Cc,
                                                      float* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int per_block = S / Cc;
  const int total = blocks * per_block;
  double s = 0.0;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int bl = i / per_block, k = c + (i - bl * per_block) * Cc;
    s += part[(size_t)bl * S + k];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = (float)red[0];
}

struct TIdx {
  int t[64];
};

// SplitMix64 (Steele, Lea and Flood, 2014): state key + (counter + 1) times
// the golden gamma, then the published finaliser
__device__ inline uint64_t splitmix64(uint64_t key, uint64_t counter) {
  uint64_t z = key + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// standard normal by the Box-Muller transform of the two 32-bit halves
// (u1 in (0, 1], u2 in [0, 1))
__device__ inline float normal_from(uint64_t r) {
  const float u1 = ((float)(uint32_t)(r >> 32) + 1.0f) * 2.3283064365386963e-10f;
  const float u2 = (float)(uint32_t)r * 2.3283064365386963e-10f;
  return sqrtf(-2.f * logf(u1)) * cosf(6.2831853071795865f * u2);
}

// network input and target from raw planes [n][3][P]: x = (q_t, q_{t-s}, 0),
// target = q_{t+s} - q_t (s the keyframe stride), q = (plane - mean) / std. With noise_std > 0 the
// inputs carry Gaussian noise (counter (b P + p) 6 + channel, key `key`) and
// the target is taken from the noisy q_t (the network learns to return to
// the data: q_t + eps + delta = q_{t+1})
__global__ void k_input_planes(const float* __restrict__ planes, int P, int nz, int stride, TIdx idx, int B,
                               float3 mean, float3 istd, float noise_std, uint64_t key, bf16* __restrict__ x,
                               float* __restrict__ target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P, p = i - b * P;
  const int t = idx.t[b];
  const float mu[3] = {mean.x, mean.y, mean.z}, is[3] = {istd.x, istd.y, istd.z};
  float qt[3], qp[3], qn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    qt[c] = (planes[((size_t)t * 3 + c) * P + p] - mu[c]) * is[c];
    qp[c] = (planes[((size_t)(t - stride) * 3 + c) * P + p] - mu[c]) * is[c];
    qn[c] = (planes[((size_t)(t + stride) * 3 + c) * P + p] - mu[c]) * is[c];
  }
  if (noise_std > 0.f) {
    const uint64_t base = (uint64_t)i * 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      qt[c] += noise_std * normal_from(splitmix64(key, base + c));
      qp[c] += noise_std * normal_from(splitmix64(key, base + 3 + c));
    }
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
  const size_t row = (size_t)i / nz;
  const int z = i - (int)(row * nz);
  store_granule(x, row, 0, z, 16, nz, r0);
  store_granule(x, row, 1, z, 16, nz, r1);
}

// pushforward inputs (after a forward pass on (q_{t-s}, q_{t-2s}) whose
// delta is in `delta`): the network's own prediction q^_t = q_{t-s} + delta
// takes the place of q_t, the previous keyframe is q_{t-s}, and the target
// is q_{t+s} - q^_t, so the network learns to correct its own one-step
// errors (no gradient flows into the first pass)
__global__ void k_pushforward_planes(const float* __restrict__ planes, int P, int nz, int stride, TIdx idx, int B,
                                     float3 mean, float3 istd, const float* __restrict__ delta,
                                     bf16* __restrict__ x, float* __restrict__ target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P, p = i - b * P;
  const int t = idx.t[b];
  const float mu[3] = {mean.x, mean.y, mean.z}, is[3] = {istd.x, istd.y, istd.z};
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
    const float qp = (planes[((size_t)(t - stride) * 3 + c) * P + p] - mu[c]) * is[c];
    const float qn = (planes[((size_t)(t + stride) * 3 + c) * P + p] - mu[c]) * is[c];
    const float qh = qp + delta[(size_t)i * 3 + c];
    e0[c] = __float2bfloat16_rn(qh);
    e0[3 + c] = __float2bfloat16_rn(qp);
    target[(size_t)i * 3 + c] = qn - qh;
  }
  const size_t row = (size_t)i / nz;
  const int z = i - (int)(row * nz);
  store_granule(x, row, 0, z, 16, nz, r0);
  store_granule(x, row, 1, z, 16, nz, r1);
}

// network input from normalised planes [B][P][3]
__global__ void k_input_q(const float* __restrict__ qt, const float* __restrict__ qp, int n, int nz,
                          bf16* __restrict__ x) {
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
  const size_t row = (size_t)i / nz;
  const int z = i - (int)(row * nz);
  store_granule(x, row, 0, z, 16, nz, r0);
  store_granule(x, row, 1, z, 16, nz, r1);
}

// gradient of the mean-square loss in delta (bf16, 16 channels, and FP32),
// per-block sums of the squared error
constexpr int LOSS_THREADS = 256;
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(const float* __restrict__ delta, const float* __restrict__ target,
                                                       int n, int nz, float scale, bf16* __restrict__ gd16,
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
    const size_t row = (size_t)i / nz;
    const int z = i - (int)(row * nz);
    store_granule(gd16, row, 0, z, 16, nz, r0);
    store_granule(gd16, row, 1, z, 16, nz, r1);
  }
  red[threadIdx.x] = se;
  __syncthreads();
  for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// sum of n partials in a fixed order: strided per thread, then a tree
__global__ void __launch_bounds__(256) k_sum_double(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
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

// bfloat16 B-operand images of one layer's weights (wimg_off): forward
// (rows = padded outputs Op, K = padded inputs Cp) and input gradient (taps
// flipped, rows = Cp, K = Op); zero in the padding
__global__ void k_pack(const float* __restrict__ w, int O, int Cc, int Op, int Cp, unsigned char* __restrict__ wf,
                       unsigned char* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * Op * Cp) return;
  const int tap = i / (Op * Cp), o = (i / Cp) % Op, c = i % Cp;
  const float val = (o < O && c < Cc) ? w[((size_t)tap * O + o) * Cc + c] : 0.f;
  const bf16 hv = __float2bfloat16_rn(val);
  *reinterpret_cast<bf16*>(wf + wimg_off(tap, o, c, Op, Cp)) = hv;
  if (wb) *reinterpret_cast<bf16*>(wb + wimg_off(8 - tap, c, o, Cp, Op)) = hv;
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

// planes mean + std ((1 - w) a + w b) from normalised [P][3] a, b
template <class T>
__global__ void k_emit_interp(const float* __restrict__ a, const float* __restrict__ b, int P, float w,
                              float3 dmean, float3 dstd, T* __restrict__ u, T* __restrict__ v, T* __restrict__ wv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float mu[3] = {dmean.x, dmean.y, dmean.z}, sd[3] = {dstd.x, dstd.y, dstd.z};
  T* outs[3] = {u, v, wv};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float q = (1.f - w) * a[(size_t)p * 3 + c] + w * b[(size_t)p * 3 + c];
    if (outs[c]) outs[c][p] = (T)(mu[c] + sd[c] * q);
  }
}

// relaxation of the rollout towards a reference plane (the data's time mean):
// delta -= lambda (q_t - q_ref)
__global__ void k_relax(float* __restrict__ delta, const float* __restrict__ qt, const float* __restrict__ qref,
                        int n, float lambda) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) delta[i] -= lambda * (qt[i] - qref[i]);
}

// Spectral relaxation of a new keyframe towards the data's power spectrum:
// f = q - q_ref per component and its separable 2-D Hartley transform
// H = H_y f H_z. With H1..H4 = H at (ky, kz), (ky, -kz), (-ky, kz), (-ky, -kz),
// the Fourier coefficients of the real plane are
//   F(ky, kz)  = (H2 + H3) / 2 - i (H1 - H4) / 2,
//   F(ky, -kz) = (H1 + H4) / 2 - i (H2 - H3) / 2,
// so each is multiplied by its factor (S(k) / |F(k)|^2)^(lambda / 2), clamped
// to [1/2, 2] per keyframe, and H1 rebuilt as f2 Re F(ky, -kz) - f1 Im F(ky, kz);
// the same transform / (ny nz) returns the relaxed plane. The phases (the
// network's structure) are kept; only the amplitude of each wavenumber moves
// towards the record's mean.
__global__ void k_spec_gather(const float* __restrict__ q, const float* __restrict__ qref, int P,
                              float* __restrict__ f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) f[(size_t)c * P + p] = q[(size_t)p * 3 + c] - qref[(size_t)p * 3 + c];
}

__device__ inline float spec_factor(float target, float pw, float lambda) {
  return (pw > 0.f && target > 0.f) ? fminf(2.f, fmaxf(0.5f, powf(target / pw, 0.5f * lambda))) : 1.f;
}

__global__ void k_spec_scale(const float* __restrict__ H, const float* __restrict__ S, int ny, int nz, float lambda,
                             float* __restrict__ out) {
  const int P = ny * nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * P) return;
  const int c = i / P, p = i - c * P;
  const int ky = p / nz, kz = p - ky * nz;
  const int my = (ny - ky) % ny, mz = (nz - kz) % nz;
  const float* Hc = H + (size_t)c * P;
  const float h1 = Hc[p], h2 = Hc[ky * nz + mz], h3 = Hc[my * nz + kz], h4 = Hc[my * nz + mz];
  const float re1 = 0.5f * (h2 + h3), im1 = -0.5f * (h1 - h4);
  const float re2 = 0.5f * (h1 + h4), im2 = -0.5f * (h2 - h3);
  const float f1 = spec_factor(S[i], re1 * re1 + im1 * im1, lambda);
  const float f2 = spec_factor(S[(size_t)c * P + ky * nz + mz], re2 * re2 + im2 * im2, lambda);
  out[i] = f2 * re2 - f1 * im1;
}

template <class T>
__global__ void k_spec_scatter(const float* __restrict__ f, const float* __restrict__ qref, int P, float inv_n,
                               float3 dmean, float3 dstd, float* __restrict__ q, T* __restrict__ u,
                               T* __restrict__ v, T* __restrict__ w) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float mu[3] = {dmean.x, dmean.y, dmean.z}, sd[3] = {dstd.x, dstd.y, dstd.z};
  T* outs[3] = {u, v, w};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float qn = qref[(size_t)p * 3 + c] + f[(size_t)c * P + p] * inv_n;
    q[(size_t)p * 3 + c] = qn;
    if (outs[c]) outs[c][p] = (T)(mu[c] + sd[c] * qn);
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
  cudaFuncSetAttribute(k_conv<N, KC, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ConvCfg<N, KC, 128>::SMEM);
  cudaFuncSetAttribute(k_conv<N, KC, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ConvCfg<N, KC, 256>::SMEM);
}
template <int NB>
void set_wgrad_attr() {
  cudaFuncSetAttribute(k_wgrad<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WgCfg<NB>::SMEM);
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// tiles of 256 pixels when the row allows, else 128; one persistent CTA per SM
template <int N, int KC>
void launch_conv(const ConvArgs& a, cudaStream_t s) {
  const int sms = num_sms();
  if (a.nz % 256 == 0) {
    const int tiles = a.rows * (a.nz / 256);
    k_conv<N, KC, 256><<<std::min(tiles, sms), CV_THREADS, ConvCfg<N, KC, 256>::SMEM, s>>>(a);
  } else {
    const int tiles = a.rows * (a.nz / 128);
    k_conv<N, KC, 128><<<std::min(tiles, sms), CV_THREADS, ConvCfg<N, KC, 128>::SMEM, s>>>(a);
  }
}

template <int NB>
void launch_wgrad(const WgArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, cudaStream_t s) {
  k_wgrad<NB><<<dim3(a.chunks, 3), WG_THREADS, WgCfg<NB>::SMEM, s>>>(a, ma, mb);
}

constexpr int WIDTH = 128;     // channels of the residual stream
constexpr int CIN_PAD = 16;    // input channels as stored (q_t, q_{t-1}, zeros)
constexpr int COUT_PAD = 16;   // output channels as computed (3 used)
constexpr int WG_CHUNKS = 50;  // CTAs per tap row of the weight gradients (3 x 50 <= 152 SMs)
constexpr int SUM_BLOCKS = 152;

struct Layer {
  int O, C, Op, Cp;        // real and padded output / input channels
  size_t woff, boff;       // offsets of W, b in the flat parameter array
  unsigned char* wf = nullptr;   // forward B-operand image (wimg_off with Op rows, Cp inputs)
  unsigned char* wb = nullptr;   // input-gradient image (flipped taps, Cp rows, Op inputs)
};

}  // namespace

}  // namespace ibm

struct ibm_gen {
  int ny = 0, nz = 0, blocks = 0, cin = 0, batch = 0, stride = 1;
  size_t P = 0;
  cudaStream_t stream = nullptr;
  double lr = 1e-3, b1 = 0.9, b2 = 0.999, eps = 1e-8;
  long long t = 0;
  size_t np = 0;
  std::vector<ibm::Layer> layers;   // in, blocks..., out
  float *w = nullptr, *gw = nullptr, *m = nullptr, *v = nullptr;
  unsigned char* wpack = nullptr;
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
  float noise_std = 0.f;            // training-input noise (normalised units)
  float relax = 0.f;                // rollout relaxation rate towards qref, per keyframe
  float* qref = nullptr;            // normalised reference plane [P][3]
  float spec_lambda = 0.f;          // spectral relaxation exponent per keyframe
  float* spec = nullptr;            // target power spectrum of q - q_ref, [3][ny][nz]
  float* sbuf[2] = {nullptr, nullptr};   // [3][ny][nz] transform scratch
  float* twz = nullptr;             // 256-point twiddles of the transform
  unsigned long long noise_seed = 0;
  int* error = nullptr;
  std::vector<void*> allocs;
  // tensor maps of the bfloat16 maps: per base address, boxes of 128 and 130 pixels
  std::vector<const void*> map_base;
  std::vector<CUtensorMap> map_box;   // 2 per base: [128-pixel box, 130-pixel box]
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

bf16* act_map(ibm_gen* g, int l) {
  return g->act + (size_t)l * ibm::map_elems((size_t)g->batch * g->ny, ibm::WIDTH, g->nz);
}

// 3-D tensor maps over a C-channel granule map: (8 channels, nz + 2 slots,
// rows x C/8 groups), boxes (8, 128 or 130 pixels, C/8 groups)
bool add_maps(ibm_gen* g, const bf16* base, int C) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t rows = (cuuint64_t)g->batch * g->ny;
  const cuuint64_t dims[3] = {8, (cuuint64_t)g->nz + 2, rows * (C / 8)};
  const cuuint64_t strides[2] = {16, ((cuuint64_t)g->nz + 2) * 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int halo = 0; halo < 2; ++halo) {
    const cuuint32_t box[3] = {8, (cuuint32_t)(ibm::WG_KP + 2 * halo), (cuuint32_t)(C / 8)};
    CUtensorMap m;
    if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    g->map_box.push_back(m);
  }
  g->map_base.push_back(base);
  return true;
}

const CUtensorMap& tmap(const ibm_gen* g, const bf16* base, bool halo) {
  size_t i = 0;
  while (i + 1 < g->map_base.size() && g->map_base[i] != base) ++i;
  return g->map_box[2 * i + (halo ? 1 : 0)];
}

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
  ConvArgs a{};
  a.ny = g->ny; a.nz = g->nz; a.rows = rows; a.error = g->error;
  // h_1 = conv(W_in, x) + b_in; act_0 = phi(h_1)
  a.in = g->x; a.w = g->layers[0].wf; a.bias = g->w + g->layers[0].boff; a.nbias = WIDTH;
  a.out32 = g->h[0]; a.ld32 = WIDTH; a.n32 = WIDTH; a.out16 = act_map(g, 0); a.out16_phi = 1;
  launch_conv<WIDTH, CIN_PAD>(a, g->stream);
  for (int l = 1; l <= g->blocks; ++l) {
    const Layer& L = g->layers[l];
    ConvArgs c = a;
    c.in = act_map(g, l - 1); c.w = L.wf; c.bias = g->w + L.boff;
    c.res = g->h[(l - 1) & 1]; c.out32 = g->h[l & 1]; c.out16 = act_map(g, l);
    launch_conv<WIDTH, WIDTH>(c, g->stream);
  }
  const Layer& Lo = g->layers.back();
  ConvArgs o{};
  o.ny = g->ny; o.nz = g->nz; o.rows = rows; o.error = g->error;
  o.in = act_map(g, g->blocks); o.w = Lo.wf; o.bias = g->w + Lo.boff; o.nbias = 3;
  o.out32 = g->delta; o.ld32 = 3; o.n32 = 3;
  launch_conv<COUT_PAD, WIDTH>(o, g->stream);
}

void wgrad(ibm_gen* g, const bf16* a, const bf16* b, int nb, int shift_a, int trans, const ibm::Layer& L, int rows) {
  using namespace ibm;
  WgArgs w{};
  w.a = a; w.b = b; w.shift_a = shift_a; w.ny = g->ny; w.nz = g->nz; w.rows = rows;
  w.chunks = WG_CHUNKS; w.part = g->part; w.error = g->error;
  const CUtensorMap& ma = tmap(g, a, shift_a != 0);
  const CUtensorMap& mb = tmap(g, b, shift_a == 0);
  if (nb == WIDTH) launch_wgrad<WIDTH>(w, ma, mb, g->stream); else launch_wgrad<16>(w, ma, mb, g->stream);
  const int n = 9 * L.O * L.C;
  k_wgrad_reduce<<<(n + 255) / 256, 256, 0, g->stream>>>(g->part, WG_CHUNKS, nb, trans, L.O, L.C, g->gw + L.woff);
}

void colsum(ibm_gen* g, const float* x, size_t pixels, int C, float* out) {
  if (C % 4 == 0) {   // an FP32 stream: per-row partials, then per channel over the rows
    const int rows = (int)(pixels / g->nz);
    ibm::k_colsum_stream<<<rows * (C / 4), 64, 0, g->stream>>>(reinterpret_cast<const float4*>(x), g->nz, C,
                                                                g->dpart);
    ibm::k_colsum_final<<<C, 256, 0, g->stream>>>(g->dpart, rows, C, C, out);
  } else {            // C = 3: 192 threads, one channel each
    ibm::k_colsum_part<<<ibm::COLSUM_BLOCKS, 192, 0, g->stream>>>(x, pixels * C, g->dpart);
    ibm::k_colsum_final<<<C, 256, 0, g->stream>>>(g->dpart, ibm::COLSUM_BLOCKS, 192, C, out);
  }
}

// loss gradients of B samples whose input x and target are in place
void backward(ibm_gen* g, int B) {
  using namespace ibm;
  const int rows = B * g->ny;
  const size_t n = (size_t)B * g->P;
  forward(g, B);
  const int lb = (int)((n + LOSS_THREADS - 1) / LOSS_THREADS);
  k_loss<<<lb, LOSS_THREADS, 0, g->stream>>>(g->delta, g->target, (int)n, g->nz, (float)(2.0 / (3.0 * n)),
                                             g->gd16, g->gd32, g->dpart);
  k_sum_double<<<1, 256, 0, g->stream>>>(g->dpart, lb, g->dscal);
  const Layer& Lo = g->layers.back();
  // output layer: dW_out^T = sum act_L[p + tap] gd[p]; db_out; g_{L+1} = phi' * conv(Wb_out, gd)
  wgrad(g, act_map(g, g->blocks), g->gd16, 16, 1, 1, Lo, rows);
  colsum(g, g->gd32, n, 3, g->gw + Lo.boff);
  ConvArgs a{};
  a.ny = g->ny; a.nz = g->nz; a.rows = rows; a.error = g->error;
  a.in = g->gd16; a.w = Lo.wb; a.dact = act_map(g, g->blocks);
  a.out32 = g->g32[0]; a.ld32 = WIDTH; a.n32 = WIDTH; a.out16 = g->g16[0];
  launch_conv<WIDTH, COUT_PAD>(a, g->stream);
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
    launch_conv<WIDTH, WIDTH>(c, g->stream);
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
  if (cfg->ny < 1 || cfg->nz < 128 || cfg->nz % 128 != 0 || cfg->width != WIDTH || cfg->blocks < 0 ||
      cfg->blocks > 64 || cfg->in_channels < 1 || cfg->in_channels > 6 || cfg->batch < 1 || cfg->batch > 64)
    return IBM_EINVAL;
  if ((size_t)cfg->ny * cfg->nz > (size_t)1 << 24) return IBM_EINVAL;
  ibm_gen* g = new (std::nothrow) ibm_gen();
  if (!g) return IBM_ENOMEM;
  g->ny = cfg->ny; g->nz = cfg->nz; g->blocks = cfg->blocks; g->cin = cfg->in_channels; g->batch = cfg->batch;
  g->stride = cfg->stride > 0 ? cfg->stride : 1;
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
  for (auto& L : g->layers) npack += wimg_bytes(L.Op, L.Cp) + wimg_bytes(L.Cp, L.Op);
  const size_t BP = (size_t)g->batch * g->P;
  const size_t rows = (size_t)g->batch * g->ny;
  bool ok = ready_attr();
  ok = ok && dalloc(g, &g->w, g->np) && dalloc(g, &g->gw, g->np) && dalloc(g, &g->m, g->np) &&
       dalloc(g, &g->v, g->np) && dalloc(g, &g->wpack, npack) && dalloc(g, &g->x, map_elems(rows, CIN_PAD, g->nz)) &&
       dalloc(g, &g->act, (size_t)(g->blocks + 1) * map_elems(rows, WIDTH, g->nz)) &&
       dalloc(g, &g->g16[0], map_elems(rows, WIDTH, g->nz)) && dalloc(g, &g->g16[1], map_elems(rows, WIDTH, g->nz)) &&
       dalloc(g, &g->gd16, map_elems(rows, COUT_PAD, g->nz)) && dalloc(g, &g->h[0], BP * WIDTH) &&
       dalloc(g, &g->h[1], BP * WIDTH) && dalloc(g, &g->g32[0], BP * WIDTH) && dalloc(g, &g->g32[1], BP * WIDTH) &&
       dalloc(g, &g->delta, BP * 3) && dalloc(g, &g->target, BP * 3) && dalloc(g, &g->gd32, BP * 3) &&
       dalloc(g, &g->part, (size_t)3 * WG_CHUNKS * 3 * 128 * WIDTH) &&
       dalloc(g, &g->dpart, (size_t)std::max<size_t>(COLSUM_BLOCKS * 1024, BP / LOSS_THREADS + 1)) &&
       dalloc(g, &g->dscal, 8) && dalloc(g, &g->hist[0], g->P * 3) && dalloc(g, &g->hist[1], g->P * 3) &&
       dalloc(g, &g->qref, g->P * 3) && dalloc(g, &g->error, 1);
  if (!ok) {
    ibm_gen_destroy(g);
    return IBM_ENOMEM;
  }
  unsigned char* pk = g->wpack;
  for (auto& L : g->layers) {
    L.wf = pk; pk += wimg_bytes(L.Op, L.Cp);
    L.wb = pk; pk += wimg_bytes(L.Cp, L.Op);
  }
  cudaMemsetAsync(g->wpack, 0, npack, g->stream);
  cudaMemsetAsync(g->w, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->gw, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->m, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->v, 0, g->np * sizeof(float), g->stream);
  cudaMemsetAsync(g->x, 0, map_elems(rows, CIN_PAD, g->nz) * sizeof(bf16), g->stream);
  bool maps = add_maps(g, g->x, CIN_PAD) && add_maps(g, g->gd16, COUT_PAD) && add_maps(g, g->g16[0], WIDTH) &&
              add_maps(g, g->g16[1], WIDTH);
  for (int l = 0; l <= g->blocks && maps; ++l) maps = add_maps(g, act_map(g, l), WIDTH);
  if (!maps) {
    ibm_gen_destroy(g);
    return IBM_ECUDA;
  }
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
  ibm::k_input_q<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(q_t, q_prev, (int)n, g->nz, g->x);
  forward(g, batch);
  if (cudaMemcpyAsync(delta, g->delta, n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  return check_error(g);
}

int ibm_gen_grad(ibm_gen* g, const float* q_t, const float* q_prev, const float* target, int batch,
                 double* loss) {
  if (!g || !q_t || !q_prev || !target || batch < 1 || batch > g->batch) return IBM_EINVAL;
  const size_t n = (size_t)batch * g->P;
  ibm::k_input_q<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(q_t, q_prev, (int)n, g->nz, g->x);
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
    if (t_idx[b] < g->stride || t_idx[b] + g->stride >= n_planes) return IBM_EINVAL;
    idx.t[b] = t_idx[b];
  }
  const size_t n = (size_t)batch * g->P;
  const float3 istd = make_float3(1.f / g->dstd.x, 1.f / g->dstd.y, 1.f / g->dstd.z);
  ibm::k_input_planes<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(
      planes, (int)g->P, g->nz, g->stride, idx, batch, g->dmean, istd, g->noise_std, g->noise_seed + (unsigned long long)g->t, g->x,
      g->target);
  backward(g, batch);
  adam(g);
  if (!loss) return cuda_status(cudaGetLastError());
  return read_loss(g, n, loss);
}

int ibm_gen_train_step_pushforward(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch,
                                   double* loss) {
  if (!g || !planes || !t_idx || batch < 1 || batch > g->batch) return IBM_EINVAL;
  ibm::TIdx idx{}, prev{};
  for (int b = 0; b < batch; ++b) {
    if (t_idx[b] < 2 * g->stride || t_idx[b] + g->stride >= n_planes) return IBM_EINVAL;
    idx.t[b] = t_idx[b];
    prev.t[b] = t_idx[b] - g->stride;
  }
  const size_t n = (size_t)batch * g->P;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const float3 istd = make_float3(1.f / g->dstd.x, 1.f / g->dstd.y, 1.f / g->dstd.z);
  // the first pass predicts q_t from (q_{t-s}, q_{t-2s}), with the training-input noise
  ibm::k_input_planes<<<nb, 256, 0, g->stream>>>(planes, (int)g->P, g->nz, g->stride, prev, batch, g->dmean, istd,
                                                 g->noise_std, g->noise_seed + (unsigned long long)g->t, g->x,
                                                 g->target);
  forward(g, batch);
  ibm::k_pushforward_planes<<<nb, 256, 0, g->stream>>>(planes, (int)g->P, g->nz, g->stride, idx, batch, g->dmean,
                                                       istd, g->delta, g->x, g->target);
  backward(g, batch);
  adam(g);
  if (!loss) return cuda_status(cudaGetLastError());
  return read_loss(g, n, loss);
}

int ibm_gen_eval(ibm_gen* g, const float* planes, int n_planes, const int* t_idx, int batch, double* loss) {
  if (!g || !planes || !t_idx || !loss || batch < 1 || batch > g->batch) return IBM_EINVAL;
  ibm::TIdx idx{};
  for (int b = 0; b < batch; ++b) {
    if (t_idx[b] < g->stride || t_idx[b] + g->stride >= n_planes) return IBM_EINVAL;
    idx.t[b] = t_idx[b];
  }
  const size_t n = (size_t)batch * g->P;
  const float3 istd = make_float3(1.f / g->dstd.x, 1.f / g->dstd.y, 1.f / g->dstd.z);
  ibm::k_input_planes<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(planes, (int)g->P, g->nz, g->stride,
                                                                          idx, batch, g->dmean, istd, 0.f, 0ull, g->x,
                                                                          g->target);
  forward(g, batch);
  const int lb = (int)((n + ibm::LOSS_THREADS - 1) / ibm::LOSS_THREADS);
  ibm::k_loss<<<lb, ibm::LOSS_THREADS, 0, g->stream>>>(g->delta, g->target, (int)n, g->nz,
                                                       (float)(2.0 / (3.0 * n)), g->gd16, g->gd32, g->dpart);
  ibm::k_sum_double<<<1, 256, 0, g->stream>>>(g->dpart, lb, g->dscal);
  return read_loss(g, n, loss);
}

int ibm_gen_set_noise(ibm_gen* g, double std, unsigned long long seed) {
  if (!g || !(std >= 0.0) || !std::isfinite(std)) return IBM_EINVAL;
  g->noise_std = (float)std;
  g->noise_seed = seed;
  return IBM_OK;
}

int ibm_gen_set_spectrum(ibm_gen* g, const double* power, double lambda) {
  if (!g || !(lambda >= 0.0 && lambda <= 1.0) || (lambda > 0.0 && !power)) return IBM_EINVAL;
  if (lambda > 0.0 && (g->ny != 256 || g->nz != 256 || !(g->relax > 0.f))) return IBM_EINVAL;
  g->spec_lambda = (float)lambda;
  if (lambda == 0.0) return IBM_OK;
  const size_t P = g->P;
  if (!g->spec) {
    if (!dalloc(g, &g->spec, 3 * P) || !dalloc(g, &g->sbuf[0], 3 * P) || !dalloc(g, &g->sbuf[1], 3 * P) ||
        !dalloc(g, &g->twz, 256))
      return IBM_ENOMEM;
    ibm::poisson_set_attributes();
  }
  std::vector<float> sp(3 * P), tw(256);
  for (size_t i = 0; i < 3 * P; ++i) sp[i] = (float)power[i];
  for (int t = 0; t < 128; ++t) {
    tw[2 * t] = (float)std::cos(2.0 * M_PI * t / 256.0);
    tw[2 * t + 1] = (float)-std::sin(2.0 * M_PI * t / 256.0);
  }
  if (cudaMemcpyAsync(g->spec, sp.data(), 3 * P * sizeof(float), cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
      cudaMemcpyAsync(g->twz, tw.data(), 256 * sizeof(float), cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return IBM_ECUDA;
  return check_error(g);
}

int ibm_gen_set_relax(ibm_gen* g, const double* plane, double lambda) {
  if (!g || !(lambda >= 0.0 && lambda <= 1.0) || (lambda > 0.0 && !plane)) return IBM_EINVAL;
  g->relax = (float)lambda;
  if (lambda == 0.0) return IBM_OK;
  const size_t P = g->P;
  std::vector<float> q(P * 3);
  const float mu[3] = {g->dmean.x, g->dmean.y, g->dmean.z}, sd[3] = {g->dstd.x, g->dstd.y, g->dstd.z};
  for (int c = 0; c < 3; ++c)
    for (size_t p = 0; p < P; ++p) q[p * 3 + c] = (float)((plane[c * P + p] - mu[c]) / sd[c]);
  if (cudaMemcpyAsync(g->qref, q.data(), P * 3 * sizeof(float), cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
    return IBM_ECUDA;
  return check_error(g);
}

int ibm_gen_set_lr(ibm_gen* g, double lr) {
  if (!g || !(lr > 0.0)) return IBM_EINVAL;
  g->lr = lr;
  return IBM_OK;
}

int ibm_gen_time(ibm_gen* g, int what, int nrep, double* ms) {
  using namespace ibm;
  if (!g || !ms || nrep < 1 || what < 0 || what > 4) return IBM_EINVAL;
  if (what >= 2 && g->blocks < 1) return IBM_EINVAL;
  const int B = g->batch, rows = B * g->ny;
  auto run = [&]() {
    switch (what) {
      case 0: backward(g, B); adam(g); break;   // training step on the data in place
      case 1: forward(g, B); break;
      case 2: {                                  // one residual-block convolution, forward
        ConvArgs c{};
        c.ny = g->ny; c.nz = g->nz; c.rows = rows; c.error = g->error;
        c.in = act_map(g, 0); c.w = g->layers[1].wf; c.bias = g->w + g->layers[1].boff; c.nbias = WIDTH;
        c.res = g->h[0]; c.out32 = g->h[1]; c.ld32 = WIDTH; c.n32 = WIDTH; c.out16 = act_map(g, 1); c.out16_phi = 1;
        launch_conv<WIDTH, WIDTH>(c, g->stream);
        break;
      }
      case 3: {                                  // its input gradient
        ConvArgs c{};
        c.ny = g->ny; c.nz = g->nz; c.rows = rows; c.error = g->error;
        c.in = g->g16[0]; c.w = g->layers[1].wb; c.dact = act_map(g, 0); c.res = g->g32[0];
        c.out32 = g->g32[1]; c.ld32 = WIDTH; c.n32 = WIDTH; c.out16 = g->g16[1];
        launch_conv<WIDTH, WIDTH>(c, g->stream);
        break;
      }
      case 4: wgrad(g, g->g16[0], act_map(g, 0), WIDTH, 0, 0, g->layers[1], rows); break;
    }
  };
  run();   // warm-up
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return IBM_ECUDA;
  cudaEventRecord(e0, g->stream);
  for (int r = 0; r < nrep; ++r) run();
  cudaEventRecord(e1, g->stream);
  const int st = check_error(g);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != IBM_OK) return st;
  *ms = (double)t / nrep;
  return IBM_OK;
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
  k_input_q<<<(P + 255) / 256, 256, 0, g->stream>>>(qt, qp, P, g->nz, g->x);
  forward(g, 1);
  if (g->relax > 0.f) k_relax<<<(3 * P + 255) / 256, 256, 0, g->stream>>>(g->delta, qt, g->qref, 3 * P, g->relax);
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
  if (g->spec_lambda > 0.f) {
    const unsigned nb = (unsigned)((P + 255) / 256);
    k_spec_gather<<<nb, 256, 0, g->stream>>>(qp, g->qref, P, g->sbuf[0]);
    if (!dht2d_planes_fp32(g->sbuf[0], g->sbuf[1], 3, g->twz, g->stream)) return IBM_ECUDA;
    k_spec_scale<<<(3 * P + 255) / 256, 256, 0, g->stream>>>(g->sbuf[1], g->spec, g->ny, g->nz, g->spec_lambda,
                                                              g->sbuf[0]);
    if (!dht2d_planes_fp32(g->sbuf[0], g->sbuf[1], 3, g->twz, g->stream)) return IBM_ECUDA;
    const float inv_n = 1.f / (float)P;
    if (precision == IBM_FP64)
      k_spec_scatter<double><<<nb, 256, 0, g->stream>>>(g->sbuf[1], g->qref, P, inv_n, g->dmean, g->dstd, qp,
                                                       (double*)u, (double*)v, (double*)w);
    else
      k_spec_scatter<float><<<nb, 256, 0, g->stream>>>(g->sbuf[1], g->qref, P, inv_n, g->dmean, g->dstd, qp,
                                                      (float*)u, (float*)v, (float*)w);
  }
  g->cur ^= 1;
  return cuda_status(cudaGetLastError());
}

int ibm_gen_emit(ibm_gen* g, double w, void* u, void* v, void* wv, int precision) {
  using namespace ibm;
  if (!g || !(w >= 0.0 && w <= 1.0)) return IBM_EINVAL;
  if (precision != IBM_FP64 && precision != IBM_FP32 && precision != IBM_MIXED) return IBM_EINVAL;
  const int P = (int)g->P;
  const float* qt = g->hist[g->cur];
  const float* qp = g->hist[g->cur ^ 1];
  if (precision == IBM_FP64)
    k_emit_interp<double><<<(P + 255) / 256, 256, 0, g->stream>>>(qp, qt, P, (float)w, g->dmean, g->dstd,
                                                                  (double*)u, (double*)v, (double*)wv);
  else
    k_emit_interp<float><<<(P + 255) / 256, 256, 0, g->stream>>>(qp, qt, P, (float)w, g->dmean, g->dstd,
                                                                 (float*)u, (float*)v, (float*)wv);
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

// ---- checkpoints: header, then the FP32 masters, Adam moments and the
// normalisation; the configuration must match on load
struct GenCkptHeader {
  char magic[8];
  int version, ny, nz, blocks, cin, stride, pad;
  long long np, t;
  double dmean[3], dstd[3], rms[3];
};

int ibm_gen_save(ibm_gen* g, const char* path) {
  if (!g || !path) return IBM_EINVAL;
  GenCkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "IBMGEN01", 8);
  h.version = 1;
  h.ny = g->ny; h.nz = g->nz; h.blocks = g->blocks; h.cin = g->cin; h.stride = g->stride;
  h.np = (long long)g->np;
  h.t = g->t;
  const float mu[3] = {g->dmean.x, g->dmean.y, g->dmean.z}, sd[3] = {g->dstd.x, g->dstd.y, g->dstd.z};
  const double rm[3] = {g->rms.x, g->rms.y, g->rms.z};
  for (int c = 0; c < 3; ++c) {
    h.dmean[c] = mu[c];
    h.dstd[c] = sd[c];
    h.rms[c] = rm[c];
  }
  std::vector<float> buf(3 * g->np);
  if (cudaMemcpyAsync(buf.data(), g->w, g->np * sizeof(float), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
      cudaMemcpyAsync(buf.data() + g->np, g->m, g->np * sizeof(float), cudaMemcpyDeviceToHost, g->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(buf.data() + 2 * g->np, g->v, g->np * sizeof(float), cudaMemcpyDeviceToHost, g->stream) !=
          cudaSuccess)
    return IBM_ECUDA;
  const int st = check_error(g);
  if (st != IBM_OK) return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return IBM_EIO;
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                  std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  return (std::fclose(f) == 0 && ok) ? IBM_OK : IBM_EIO;
}

int ibm_gen_load(ibm_gen* g, const char* path) {
  if (!g || !path) return IBM_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return IBM_EIO;
  GenCkptHeader h;
  std::vector<float> buf(3 * g->np);
  bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, "IBMGEN01", 8) == 0 && h.version == 1;
  if (ok && (h.ny != g->ny || h.nz != g->nz || h.blocks != g->blocks || h.cin != g->cin ||
             h.stride != g->stride || h.np != (long long)g->np)) {
    std::fclose(f);
    return IBM_EINVAL;
  }
  ok = ok && std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing may follow
  std::fclose(f);
  if (!ok) return IBM_EIO;
  if (cudaMemcpyAsync(g->w, buf.data(), g->np * sizeof(float), cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
      cudaMemcpyAsync(g->m, buf.data() + g->np, g->np * sizeof(float), cudaMemcpyHostToDevice, g->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(g->v, buf.data() + 2 * g->np, g->np * sizeof(float), cudaMemcpyHostToDevice, g->stream) !=
          cudaSuccess)
    return IBM_ECUDA;
  g->t = h.t;
  g->dmean = make_float3((float)h.dmean[0], (float)h.dmean[1], (float)h.dmean[2]);
  g->dstd = make_float3((float)h.dstd[0], (float)h.dstd[1], (float)h.dstd[2]);
  g->rms = make_double3(h.rms[0], h.rms[1], h.rms[2]);
  pack_weights(g);
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
