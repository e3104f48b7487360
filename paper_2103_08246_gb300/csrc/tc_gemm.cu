// Split-TF32 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a) for
// the Hartley transforms of the mixed-precision pressure solve: for every
// n x n plane X (n = 32, 64, 128 or 256; rows of n contiguous values) it
// computes
//   out = (X H)^T,   H[k][c] = cas(2 pi k c / n) = cos + sin,
// applied twice, ((X H)^T H)^T = H X H: the 2-D transform of the plane.
//
// Planes of 256 (the production case) use the even/odd form below; planes
// of 32, 64 and 128 (the ensemble's members) the direct form (namespace
// direct), one n x n contraction per row with a lighter register footprint.
//
// Even/odd split of each row x (m = n / 2): with e[0] = x[0], o[0] = 0 and
//   e[k] = x[k] + x[n - k],  o[k] = x[k] - x[n - k]        k = 1 .. m - 1,
//   C[c] = sum_{k<m} e[k] cos(2 pi k c / n),  S[c] = sum_{k<m} o[k] sin(2 pi k c / n),
// the row's transform is
//   y[c] = C[c] + S[c] + x[m] (-1)^c,  y[n - c] = C[c] - S[c] + x[m] (-1)^c   (c < m),
//   y[m] = sum_k x[k] (-1)^k,
// two m x m contractions instead of one n x n: half the tensor-core work and
// half the bytes of the matrix operands. Operands are rounded as
// a ~ a_hi + a_lo, a_hi = tf32(a), a_lo = tf32(a - a_hi) (round to nearest,
// ties away), and a_hi b_hi + a_hi b_lo + a_lo b_hi is accumulated in FP32 in
// tensor memory.
//
// Persistent and warp-specialised, one CTA per SM, tiles of 128 rows (of one
// or several planes); stage j of a tile holds the raw K blocks j and
// n / 16 - 1 - j (16 values of every row each), so a row is read once:
//  * warp 0 (one thread) fills a stage with two tensor-map copies of raw
//    blocks, which land in the K-major core-matrix layout (box of 4 floats x
//    128 rows x 4 K-groups: [K-group][row][16 bytes]), and one bulk copy of
//    the stage's slice of the pre-split cos / sin image (tc_pack_hartley);
//  * warps 2-5 (one thread per row) form e and o of the stage's 16 K values
//    (the mirror of the block's first value is the previous stage's last
//    block's first value), write e_hi / o_hi over the raw blocks and e_lo /
//    o_lo beside them, and keep x[m] and the alternating sum of the row for
//    the epilogue;
//  * warp 1 (one thread) issues 2 x 2 x 3 tcgen05.mma (M = 128, N = m,
//    K = 8) per stage into the tile's C and S accumulators (one of two
//    tensor-memory buffers), commits them to the stage's "empty" barrier and,
//    after the tile's last stage, to the buffer's "full" barrier;
//  * warps 6-13 read the other buffer back with tcgen05.ld (warp w its lane
//    quarter w % 4, half of the columns), form y and store it transposed into
//    the plane: for every column the warp's 32 rows are 32 consecutive
//    floats. Rows past the last plane load zeros (the tensor map's
//    out-of-range fill) and store nothing.
// Every mbarrier wait is bounded; on expiry the waiting thread records it
// and carries on, the kernel sets the error flag, waits (bounded) for its own
// tensor-core work, releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "solver.h"
#include "tcgen05.cuh"

namespace ibm {

namespace {

constexpr int TC_M = 128, TC_KB = 16;
constexpr int TC_THREADS = 448;                    // 14 warps
constexpr int TC_CONV_WARPS = 4, TC_EPI_WARPS = 8;
constexpr int TC_EPI0 = 2 + TC_CONV_WARPS;         // first epilogue warp
constexpr uint32_t A_TILE = TC_M * TC_KB * 4;      // one raw block (or one e / o part): 8 KB
constexpr uint32_t A_LBO = TC_M * 16;              // K-adjacent core matrices of A
constexpr uint32_t SMEM_BUDGET = 192 * 1024;
// SPLIT = 3: the three split products (FP32-class result); SPLIT = 1: the
// single product a_hi b_hi (TF32-class, about 2^-11 relative), half the
// shared-memory bytes per stage and so twice the stages in flight
template <int N, int SPLIT = 3>
struct TcCfg {
  static constexpr int MH = N / 2;                              // m: the contractions' K and N
  static constexpr uint32_t B_PART = (uint32_t)MH * TC_KB * 4;  // one of cos_hi, cos_lo, sin_hi, sin_lo
  static constexpr uint32_t B_LBO = (uint32_t)MH * 16;
  static constexpr uint32_t B_TX = (SPLIT == 3 ? 4 : 2) * B_PART;
  // e_hi (over raw block j), o_hi (over raw block n/16-1-j), [e_lo, o_lo,] then the B parts
  static constexpr uint32_t A_PARTS = SPLIT == 3 ? 4 : 2;
  static constexpr uint32_t STAGE = A_PARTS * A_TILE + B_TX;
  static constexpr int MAX_STAGES = SPLIT == 3 ? 3 : 6;
  static constexpr int STAGES =
      SMEM_BUDGET / STAGE > MAX_STAGES ? MAX_STAGES : (int)(SMEM_BUDGET / STAGE);
  static constexpr uint32_t SMEM = STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = 4 * MH;                 // two buffers of C and S
  static constexpr int NS = N / 32;                             // stages per tile
  static constexpr int NB = N / 16;                             // raw K blocks per row
};

__device__ inline uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int N) {
  return (1u << 4)                      // D format F32
         | (2u << 7)                    // A format TF32
         | (2u << 10)                   // B format TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ inline void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// copy of the tensor-map box at (x, y, z) of a 3-D map
__device__ inline void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline void bulk_g2s_u32(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst), "l"(src),
      "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline uint4 split_hi(const float (&v)[4], uint4& lo) {
  uint4 h;
  h.x = tf32_bits(v[0]);
  h.y = tf32_bits(v[1]);
  h.z = tf32_bits(v[2]);
  h.w = tf32_bits(v[3]);
  lo.x = tf32_bits(v[0] - __uint_as_float(h.x));
  lo.y = tf32_bits(v[1] - __uint_as_float(h.y));
  lo.z = tf32_bits(v[2] - __uint_as_float(h.z));
  lo.w = tf32_bits(v[3] - __uint_as_float(h.w));
  return h;
}

struct TcArgs {
  const unsigned char* img;    // pre-split cos / sin image (tc_pack_hartley)
  float* out;                  // per plane: out[c][r] = sum_k X[r][k] H[k][c]
  int M;                       // rows of X (planes x n)
  int* error;
};

template <int N, int SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc_tf32x3(TcArgs g, const __grid_constant__ CUtensorMap xmap) {
  using C = TcCfg<N, SPLIT>;
  constexpr int MH = C::MH, ST = C::STAGES;
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t full[ST], conv[ST], empty[ST], tfull[2], tempty[2], xfull[2], xempty[2];
  __shared__ float xm_s[2][TC_M], ym_s[2][TC_M];   // per row of a tile: x[m] and y[m]
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * C::NS;
  const uint32_t sbase = smem_u32(tsm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], TC_CONV_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TC_EPI_WARPS);
      mbar_init(&xfull[b], TC_CONV_WARPS);
      mbar_init(&xempty[b], TC_EPI_WARPS);
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
        const int s = j % ST;
        if (j >= ST) ok = mbar_wait(&empty[s], (uint32_t)(j / ST - 1) & 1u) && ok;
        const int lt = j / C::NS, js = j % C::NS;
        const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M;
        const uint32_t st = sbase + (uint32_t)s * C::STAGE;
        mbar_arrive_expect_tx(&full[s], 2 * A_TILE + C::B_TX);
        tma_load_3d(st, &xmap, 0, m0, js * (TC_KB / 4), &full[s]);
        tma_load_3d(st + A_TILE, &xmap, 0, m0, (C::NB - 1 - js) * (TC_KB / 4), &full[s]);
        // the image holds cos_hi, cos_lo, sin_hi, sin_lo per stage slice
        const unsigned char* slice = g.img + (size_t)js * 4 * C::B_PART;
        if constexpr (SPLIT == 3) {
          bulk_g2s_u32(st + C::A_PARTS * A_TILE, slice, C::B_TX, &full[s]);
        } else {
          bulk_g2s_u32(st + C::A_PARTS * A_TILE, slice, C::B_PART, &full[s]);
          bulk_g2s_u32(st + C::A_PARTS * A_TILE + C::B_PART, slice + 2 * C::B_PART, C::B_PART, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(MH);
      for (int j = 0; j < total; ++j) {
        const int s = j % ST;
        const int lt = j / C::NS, js = j % C::NS;
        // the buffer's previous tile (lt - 2) must have been read out
        if (js == 0 && lt >= 2) ok = mbar_wait(&tempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        ok = mbar_wait(&conv[s], (uint32_t)(j / ST) & 1u) && ok;
        tc_fence_after();
        const uint32_t dc = tmem + (uint32_t)((lt & 1) * 2 * MH), ds = dc + (uint32_t)MH;
        const uint32_t eh = sbase + (uint32_t)s * C::STAGE, oh = eh + A_TILE, el = eh + 2 * A_TILE,
                       ol = eh + 3 * A_TILE;
        const uint32_t ch = eh + C::A_PARTS * A_TILE;
        const uint32_t cl = ch + C::B_PART, sh = SPLIT == 3 ? cl + C::B_PART : ch + C::B_PART,
                       sl = sh + C::B_PART;
#pragma unroll
        for (int kk = 0; kk < TC_KB / 8; ++kk) {   // K = 8: two K-groups per instruction
          const uint32_t ka = (uint32_t)kk * 2 * A_LBO, kb2 = (uint32_t)kk * 2 * C::B_LBO;
          const uint32_t first = (js == 0 && kk == 0) ? 0u : 1u;
          tc_mma(dc, tc_desc(eh + ka, A_LBO, 128), tc_desc(ch + kb2, C::B_LBO, 128), idesc, first);
          if constexpr (SPLIT == 3) {
            tc_mma(dc, tc_desc(eh + ka, A_LBO, 128), tc_desc(cl + kb2, C::B_LBO, 128), idesc, 1u);
            tc_mma(dc, tc_desc(el + ka, A_LBO, 128), tc_desc(ch + kb2, C::B_LBO, 128), idesc, 1u);
          }
          tc_mma(ds, tc_desc(oh + ka, A_LBO, 128), tc_desc(sh + kb2, C::B_LBO, 128), idesc, first);
          if constexpr (SPLIT == 3) {
            tc_mma(ds, tc_desc(oh + ka, A_LBO, 128), tc_desc(sl + kb2, C::B_LBO, 128), idesc, 1u);
            tc_mma(ds, tc_desc(ol + ka, A_LBO, 128), tc_desc(sh + kb2, C::B_LBO, 128), idesc, 1u);
          }
        }
        tc_commit_to(&empty[s]);
        if (js == C::NS - 1) tc_commit_to(&tfull[lt & 1]);
      }
    }
  } else if (warp < TC_EPI0) {
    // one thread per row of the tile: e and o of the stage's 16 K values
    const int t = tid - 64;
    float carry = 0.f, alt = 0.f;
    for (int j = 0; j < total; ++j) {
      const int s = j % ST;
      const int lt = j / C::NS, js = j % C::NS;
      ok = mbar_wait(&full[s], (uint32_t)(j / ST) & 1u) && ok;
      unsigned char* st = tsm + (size_t)s * C::STAGE;
      float a[16], b[16];
#pragma unroll
      for (int kg = 0; kg < 4; ++kg) {
        const float4 va = *reinterpret_cast<const float4*>(st + kg * A_LBO + t * 16);
        const float4 vb = *reinterpret_cast<const float4*>(st + A_TILE + kg * A_LBO + t * 16);
        a[4 * kg] = va.x, a[4 * kg + 1] = va.y, a[4 * kg + 2] = va.z, a[4 * kg + 3] = va.w;
        b[4 * kg] = vb.x, b[4 * kg + 1] = vb.y, b[4 * kg + 2] = vb.z, b[4 * kg + 3] = vb.w;
      }
      if (js == 0) alt = 0.f;
      float e[16], o[16];
      // the mirror n - k of k = 16 js + q is b[16 - q] (q > 0); of k = 16 js it
      // is the first value of the previous stage's second block (none for k = 0)
      e[0] = js == 0 ? a[0] : a[0] + carry;
      o[0] = js == 0 ? 0.f : a[0] - carry;
#pragma unroll
      for (int q = 1; q < 16; ++q) {
        e[q] = a[q] + b[16 - q];
        o[q] = a[q] - b[16 - q];
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) alt += (q & 1) ? -(a[q] + b[q]) : (a[q] + b[q]);
      carry = b[0];
#pragma unroll
      for (int kg = 0; kg < 4; ++kg) {
        const float ve[4] = {e[4 * kg], e[4 * kg + 1], e[4 * kg + 2], e[4 * kg + 3]};
        const float vo[4] = {o[4 * kg], o[4 * kg + 1], o[4 * kg + 2], o[4 * kg + 3]};
        uint4 lo;
        const uint4 he = split_hi(ve, lo);
        *reinterpret_cast<uint4*>(st + kg * A_LBO + t * 16) = he;
        if constexpr (SPLIT == 3) *reinterpret_cast<uint4*>(st + 2 * A_TILE + kg * A_LBO + t * 16) = lo;
        const uint4 ho = split_hi(vo, lo);
        *reinterpret_cast<uint4*>(st + A_TILE + kg * A_LBO + t * 16) = ho;
        if constexpr (SPLIT == 3) *reinterpret_cast<uint4*>(st + 3 * A_TILE + kg * A_LBO + t * 16) = lo;
      }
      fence_proxy_async_smem();   // generic-proxy writes -> visible to the tensor core
      if (js == C::NS - 1) {
        // x[m] is the first value of the last stage's second block
        if (lt >= 2) ok = mbar_wait(&xempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        xm_s[lt & 1][t] = b[0];
        ym_s[lt & 1][t] = alt;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&conv[s]);
        if (js == C::NS - 1) mbar_arrive(&xfull[lt & 1]);
      }
    }
  } else {
    // epilogue warps: lane quarter warp % 4, column half (warp - TC_EPI0) / 4
    const int quarter = warp & 3, part = (warp - TC_EPI0) >> 2;
    constexpr int SPLIT = MH >= 32 ? 2 : 1;
    constexpr int CW = MH / SPLIT < 32 ? MH / SPLIT : 32;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int r = quarter * 32 + lane;
      const int m = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M + r;
      ok = mbar_wait(&tfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      ok = mbar_wait(&xfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      tc_fence_after();
      const float xm = xm_s[lt & 1][r];
      const uint32_t dc = tmem + (uint32_t)((lt & 1) * 2 * MH) + ((uint32_t)(quarter * 32) << 16);
      float* plane = g.out + (size_t)(m / N) * N * N + (m % N);
      const bool live = m < g.M;
      if (part == 0 && live) plane[(size_t)MH * N] = ym_s[lt & 1][r];
      if (part < SPLIT) {
#pragma unroll 1
        for (int c0 = part * (MH / SPLIT); c0 < (part + 1) * (MH / SPLIT); c0 += CW) {
          float vc[CW], vs[CW];
          if constexpr (CW == 32) {
            tc_ld_x32(dc + (uint32_t)c0, vc);
            tc_ld_x32(dc + (uint32_t)(MH + c0), vs);
          } else {
            tc_ld_x16(dc + (uint32_t)c0, vc);
            tc_ld_x16(dc + (uint32_t)(MH + c0), vs);
          }
          if (live) {
#pragma unroll
            for (int q = 0; q < CW; ++q) {
              const int c = c0 + q;
              const float base = vc[q] + ((c & 1) ? -xm : xm);
              plane[(size_t)c * N] = base + vs[q];
              if (c > 0) plane[(size_t)(N - c) * N] = base - vs[q];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty[lt & 1]);
        mbar_arrive(&xempty[lt & 1]);
      }
    }
  }
  // every MMA has completed once the last tile's buffer was committed
  if (tid == 32 && my_tiles > 0)
    ok = mbar_wait(&tfull[(my_tiles - 1) & 1], (uint32_t)((my_tiles - 1) / 2) & 1u) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, C::TMEM_COLS);
}

// ---- BF16 storage at 256 x 256 planes (the refinement's correction when the
// predictor is the FP32 FFT solve): the same even/odd form with X and out in
// bfloat16, e and o rounded to bfloat16 (relative 2^-9), products
// e cos + o sin by tcgen05.mma kind::f16 (M = 128, N = 128, K = 16) into FP32
// accumulators. The whole cos / sin image (2 x 128 x 128 bfloat16, 64 KB)
// stays in shared memory for the kernel's lifetime, so a stage carries only
// the two raw K blocks (8 KB) and twelve stages are in flight. A raw block of
// 16 values is two K-groups of 8 bfloat16 (16 bytes per row of a core
// matrix); one MMA per accumulator consumes it.
namespace b16 {

constexpr int N = 256, MH = 128, NS = N / 32, NB = N / 16;
constexpr uint32_t A_TILE = TC_M * TC_KB * 2;      // one raw block of 128 rows: 4 KB
constexpr uint32_t STAGE = 2 * A_TILE;
constexpr uint32_t IMG = 2u * MH * MH * 2;         // cos, sin: 64 KB
constexpr uint32_t IMG_SLICE = 2u * TC_KB * MH * 2;   // one stage's cos + sin K-slice: 8 KB
constexpr uint32_t B_LBO = MH * 16;                // K-adjacent core matrices of a cos / sin part
constexpr int ST = 12;
constexpr uint32_t SMEM = IMG + ST * STAGE;        // 160 KB
constexpr uint32_t TMEM_COLS = 4 * MH;             // two buffers of C and S

struct Args {
  const unsigned char* img;   // tc_pack_hartley_bf16
  __nv_bfloat16* out;         // per plane: out[c][r] = sum_k X[r][k] H[k][c]
  int M;                      // rows of X (planes x 256)
  int* error;
};

__device__ inline void unpack8(uint4 v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    f[2 * q] = __uint_as_float(w[q] << 16);
    f[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
  }
}

__device__ inline uint4 pack8(const float* f) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
    w[q] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc_bf16(Args g, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t full[ST], conv[ST], empty[ST], tfull[2], tempty[2], xfull[2], xempty[2], imgbar;
  __shared__ float xm_s[2][TC_M], ym_s[2][TC_M];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * NS;
  const uint32_t ibase = smem_u32(tsm), sbase = ibase + IMG;

  if (warp == 0) tc_alloc(&tmem_slot, TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], TC_CONV_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TC_EPI_WARPS);
      mbar_init(&xfull[b], TC_CONV_WARPS);
      mbar_init(&xempty[b], TC_EPI_WARPS);
    }
    mbar_init(&imgbar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      if (total > 0) {
        mbar_arrive_expect_tx(&imgbar, IMG);
        for (uint32_t o = 0; o < IMG; o += 16384) bulk_g2s_u32(ibase + o, g.img + o, 16384, &imgbar);
      }
      for (int j = 0; j < total; ++j) {
        const int s = j % ST;
        if (j >= ST) ok = mbar_wait(&empty[s], (uint32_t)(j / ST - 1) & 1u) && ok;
        const int lt = j / NS, js = j % NS;
        const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M;
        const uint32_t st = sbase + (uint32_t)s * STAGE;
        mbar_arrive_expect_tx(&full[s], 2 * A_TILE);
        tma_load_3d(st, &xmap, 0, m0, js * (TC_KB / 8), &full[s]);
        tma_load_3d(st + A_TILE, &xmap, 0, m0, (NB - 1 - js) * (TC_KB / 8), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc_bf16(TC_M, MH, false, false);
      if (total > 0) ok = mbar_wait(&imgbar, 0u) && ok;
      for (int j = 0; j < total; ++j) {
        const int s = j % ST;
        const int lt = j / NS, js = j % NS;
        if (js == 0 && lt >= 2) ok = mbar_wait(&tempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        ok = mbar_wait(&conv[s], (uint32_t)(j / ST) & 1u) && ok;
        tc_fence_after();
        const uint32_t dc = tmem + (uint32_t)((lt & 1) * 2 * MH), ds = dc + (uint32_t)MH;
        const uint32_t e = sbase + (uint32_t)s * STAGE, o = e + A_TILE;
        const uint32_t cs = ibase + (uint32_t)js * IMG_SLICE, sn = cs + IMG_SLICE / 2;
        const uint32_t first = js == 0 ? 0u : 1u;
        tc_mma_bf16(dc, tc_desc(e, A_LBO, 128), tc_desc(cs, B_LBO, 128), idesc, first);
        tc_mma_bf16(ds, tc_desc(o, A_LBO, 128), tc_desc(sn, B_LBO, 128), idesc, first);
        tc_commit_to(&empty[s]);
        if (js == NS - 1) tc_commit_to(&tfull[lt & 1]);
      }
    }
  } else if (warp < TC_EPI0) {
    const int t = tid - 64;   // the tile row this thread converts
    float carry = 0.f, alt = 0.f;
    for (int j = 0; j < total; ++j) {
      const int s = j % ST;
      const int lt = j / NS, js = j % NS;
      ok = mbar_wait(&full[s], (uint32_t)(j / ST) & 1u) && ok;
      unsigned char* st = tsm + IMG + (size_t)s * STAGE;
      float a[16], b[16];
#pragma unroll
      for (int kg = 0; kg < 2; ++kg) {
        unpack8(*reinterpret_cast<const uint4*>(st + kg * A_LBO + t * 16), a + 8 * kg);
        unpack8(*reinterpret_cast<const uint4*>(st + A_TILE + kg * A_LBO + t * 16), b + 8 * kg);
      }
      if (js == 0) alt = 0.f;
      float ev[16], ov[16];
      ev[0] = js == 0 ? a[0] : a[0] + carry;
      ov[0] = js == 0 ? 0.f : a[0] - carry;
#pragma unroll
      for (int q = 1; q < 16; ++q) {
        ev[q] = a[q] + b[16 - q];
        ov[q] = a[q] - b[16 - q];
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) alt += (q & 1) ? -(a[q] + b[q]) : (a[q] + b[q]);
      carry = b[0];
#pragma unroll
      for (int kg = 0; kg < 2; ++kg) {
        *reinterpret_cast<uint4*>(st + kg * A_LBO + t * 16) = pack8(ev + 8 * kg);
        *reinterpret_cast<uint4*>(st + A_TILE + kg * A_LBO + t * 16) = pack8(ov + 8 * kg);
      }
      fence_proxy_async_smem();
      if (js == NS - 1) {
        if (lt >= 2) ok = mbar_wait(&xempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        xm_s[lt & 1][t] = b[0];
        ym_s[lt & 1][t] = alt;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&conv[s]);
        if (js == NS - 1) mbar_arrive(&xfull[lt & 1]);
      }
    }
  } else {
    // epilogue: lane quarter warp % 4, column half (warp - TC_EPI0) / 4
    const int quarter = warp & 3, part = (warp - TC_EPI0) >> 2;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int r = quarter * 32 + lane;
      const int m = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M + r;
      ok = mbar_wait(&tfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      ok = mbar_wait(&xfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      tc_fence_after();
      const float xm = xm_s[lt & 1][r];
      const uint32_t dc = tmem + (uint32_t)((lt & 1) * 2 * MH) + ((uint32_t)(quarter * 32) << 16);
      __nv_bfloat16* plane = g.out + (size_t)(m / N) * N * N + (m % N);
      const bool live = m < g.M;
      if (part == 0 && live) plane[(size_t)MH * N] = __float2bfloat16_rn(ym_s[lt & 1][r]);
#pragma unroll 1
      for (int c0 = part * (MH / 2); c0 < (part + 1) * (MH / 2); c0 += 32) {
        float vc[32], vs[32];
        tc_ld_x32(dc + (uint32_t)c0, vc);
        tc_ld_x32(dc + (uint32_t)(MH + c0), vs);
        if (live) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int c = c0 + q;
            const float base = vc[q] + ((c & 1) ? -xm : xm);
            plane[(size_t)c * N] = __float2bfloat16_rn(base + vs[q]);
            if (c > 0) plane[(size_t)(N - c) * N] = __float2bfloat16_rn(base - vs[q]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty[lt & 1]);
        mbar_arrive(&xempty[lt & 1]);
      }
    }
  }
  if (tid == 32 && my_tiles > 0)
    ok = mbar_wait(&tfull[(my_tiles - 1) & 1], (uint32_t)((my_tiles - 1) / 2) & 1u) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, TMEM_COLS);
}

// image: per stage slice js (K = 16 js .. 16 js + 15), cos then sin, each as
// [K-group (2)][c (128)][8 bfloat16]
__global__ void k_pack(uint16_t* __restrict__ img) {
  const int total = 2 * MH * MH;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int e = i & 7;
    const int c = (i >> 3) & (MH - 1);
    const int rest = i >> 10;   // (js * 2 + part) * 2 + kg
    const int kg = rest & 1, part = (rest >> 1) & 1, js = rest >> 2;
    const int k = js * TC_KB + kg * 8 + e;
    const int kc = (k * c) % N;
    double sv, cv;
    sincospi(2.0 * (double)kc / (double)N, &sv, &cv);
    const __nv_bfloat16 h = __float2bfloat16_rn((float)(part == 0 ? cv : sv));
    img[i] = *reinterpret_cast<const uint16_t*>(&h);
  }
}

}  // namespace b16

// ---- direct form for planes of 32, 64 and 128 (the ensemble's members): one
// n x n contraction per row, K in blocks of 16 through a four-stage ring, the
// A block split in place by six warps; 512 threads at about 53 registers
// leave room on the SM for the concurrent kernels of other ensemble members
// (the even/odd form above holds 448 threads at 128 registers)
namespace direct {

constexpr int D_STAGES = 4;
constexpr int D_THREADS = 512;                     // 16 warps
constexpr int D_CONV_WARPS = 6, D_EPI_WARPS = 8;
template <int N>
struct DCfg {
  static constexpr uint32_t B_TILE = (uint32_t)N * TC_KB * 4;
  static constexpr uint32_t B_LBO = (uint32_t)N * 16;
  static constexpr uint32_t STAGE = 2 * A_TILE + 2 * B_TILE;   // A_hi, A_lo, B_hi, B_lo
  static constexpr uint32_t SMEM = D_STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = 2 * N;                 // two accumulators
  static constexpr int NKB = N / TC_KB;
};

struct DArgs {
  const unsigned char* himg;   // pre-split H (k_pack_direct)
  float* out;                  // per plane: out[c][r] = sum_k X[r][k] H[k][c]
  int M;                       // rows of X (planes x n)
  int* error;
};

template <int N>
__global__ void __launch_bounds__(D_THREADS, 1) k_gemm_tc_direct(DArgs g, const __grid_constant__ CUtensorMap xmap) {
  using C = DCfg<N>;
  constexpr uint32_t A_TX = A_TILE, B_TX = 2 * C::B_TILE;
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t full[D_STAGES], conv[D_STAGES], empty[D_STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * C::NKB;
  const uint32_t sbase = smem_u32(tsm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < D_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], D_CONV_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], D_EPI_WARPS);
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
        const int s = j % D_STAGES;
        if (j >= D_STAGES) ok = mbar_wait(&empty[s], (uint32_t)(j / D_STAGES - 1) & 1u) && ok;
        const int lt = j / C::NKB, kb = j % C::NKB;
        const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M;
        const uint32_t st = sbase + (uint32_t)s * C::STAGE;
        mbar_arrive_expect_tx(&full[s], A_TX + B_TX);
        tma_load_3d(st, &xmap, 0, m0, kb * (TC_KB / 4), &full[s]);
        bulk_g2s_u32(st + 2 * A_TILE, g.himg + (size_t)kb * B_TX, B_TX, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(N);
      for (int j = 0; j < total; ++j) {
        const int s = j % D_STAGES;
        const int lt = j / C::NKB, kb = j % C::NKB;
        // the accumulator's previous tile (lt - 2) must have been read out
        if (kb == 0 && lt >= 2) ok = mbar_wait(&tempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        ok = mbar_wait(&conv[s], (uint32_t)(j / D_STAGES) & 1u) && ok;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)((lt & 1) * N);
        const uint32_t ah = sbase + (uint32_t)s * C::STAGE, al = ah + A_TILE;
        const uint32_t bh = ah + 2 * A_TILE, bl = bh + C::B_TILE;
#pragma unroll
        for (int kk = 0; kk < TC_KB / 8; ++kk) {   // K = 8: two K-groups per instruction
          const uint32_t ka = (uint32_t)kk * 2 * A_LBO, kb2 = (uint32_t)kk * 2 * C::B_LBO;
          tc_mma(d, tc_desc(ah + ka, A_LBO, 128), tc_desc(bh + kb2, C::B_LBO, 128), idesc,
                 (kb == 0 && kk == 0) ? 0u : 1u);
          tc_mma(d, tc_desc(ah + ka, A_LBO, 128), tc_desc(bl + kb2, C::B_LBO, 128), idesc, 1u);
          tc_mma(d, tc_desc(al + ka, A_LBO, 128), tc_desc(bh + kb2, C::B_LBO, 128), idesc, 1u);
        }
        tc_commit_to(&empty[s]);
        if (kb == C::NKB - 1) tc_commit_to(&tfull[lt & 1]);
      }
    }
  } else if (warp < 2 + D_CONV_WARPS) {
    // split: 16-byte chunks of the A block, a_hi in place, a_lo to the second tile
    const int ct = tid - 64;
    constexpr int CHUNKS = A_TILE / 16;
    for (int j = 0; j < total; ++j) {
      const int s = j % D_STAGES;
      ok = mbar_wait(&full[s], (uint32_t)(j / D_STAGES) & 1u) && ok;
      uint4* hi = reinterpret_cast<uint4*>(tsm + (size_t)s * C::STAGE);
      uint4* lo = reinterpret_cast<uint4*>(tsm + (size_t)s * C::STAGE + A_TILE);
      for (int q = ct; q < CHUNKS; q += 32 * D_CONV_WARPS) {
        const uint4 v = hi[q];
        uint4 h, l;
        h.x = tf32_bits(__uint_as_float(v.x));
        h.y = tf32_bits(__uint_as_float(v.y));
        h.z = tf32_bits(__uint_as_float(v.z));
        h.w = tf32_bits(__uint_as_float(v.w));
        l.x = tf32_bits(__uint_as_float(v.x) - __uint_as_float(h.x));
        l.y = tf32_bits(__uint_as_float(v.y) - __uint_as_float(h.y));
        l.z = tf32_bits(__uint_as_float(v.z) - __uint_as_float(h.z));
        l.w = tf32_bits(__uint_as_float(v.w) - __uint_as_float(h.w));
        hi[q] = h;
        lo[q] = l;
      }
      fence_proxy_async_smem();   // generic-proxy writes -> visible to the tensor core
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
    }
  } else {
    // epilogue warps 8 .. 15: lane quarter warp % 4, column half (warp - 8) / 4
    const int quarter = warp & 3, part = (warp - 8) >> 2;
    constexpr int SPLIT = N >= 64 ? 2 : 1;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int m = ((int)blockIdx.x + lt * (int)gridDim.x) * TC_M + quarter * 32 + lane;
      ok = mbar_wait(&tfull[lt & 1], (uint32_t)(lt / 2) & 1u) && ok;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)((lt & 1) * N) + ((uint32_t)(quarter * 32) << 16);
      float* plane = g.out + (size_t)(m / N) * N * N + (m % N);
      if (part < SPLIT) {
#pragma unroll 1
        for (int c0 = part * (N / SPLIT); c0 < (part + 1) * (N / SPLIT); c0 += 32) {
          float v[32];
          tc_ld_x32(d + (uint32_t)c0, v);
          if (m < g.M) {
#pragma unroll
            for (int q = 0; q < 32; ++q) plane[(size_t)(c0 + q) * N] = v[q];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[lt & 1]);
    }
  }
  // every MMA has completed once the last tile's accumulator was committed
  if (tid == 32 && my_tiles > 0)
    ok = mbar_wait(&tfull[(my_tiles - 1) & 1], (uint32_t)((my_tiles - 1) / 2) & 1u) && ok;
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, C::TMEM_COLS);
}

// pre-split H image: per K block kb, the hi tile then the lo tile, each
// [K-group][n][4 floats], element (c, k) = cas(2 pi (k c mod n) / n) from
// FP64 sincospi; hi = tf32(v), lo = tf32(v - hi) with the remainder in FP64
__global__ void k_pack_direct(int n, uint32_t* __restrict__ img) {
  const int total = 2 * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int e = i & 3;
    const int c = (i >> 2) % n;
    const int rest = (i >> 2) / n;              // (kb * 2 + part) * (TC_KB / 4) + kg
    const int kg = rest % (TC_KB / 4);
    const int part = (rest / (TC_KB / 4)) & 1;
    const int kb = rest / (2 * (TC_KB / 4));
    const int k = kb * TC_KB + kg * 4 + e;
    const long long kc = ((long long)k * c) % n;
    double sv, cv;
    sincospi(2.0 * (double)kc / (double)n, &sv, &cv);
    const double v = cv + sv;
    const uint32_t h = tf32_bits((float)v);
    img[i] = part == 0 ? h : tf32_bits((float)(v - (double)__uint_as_float(h)));
  }
}

}  // namespace direct

// pre-split cos / sin image: per stage js (K rows k = 16 js .. 16 js + 15),
// the parts cos_hi, cos_lo, sin_hi, sin_lo, each [K-group][c][4 floats],
// c < n / 2, element (c, k) = cos or sin of 2 pi (k c mod n) / n from FP64
// sincospi; hi = tf32(v), lo = tf32(v - hi) with the remainder taken in FP64
__global__ void k_pack_hartley(int n, uint32_t* __restrict__ img) {
  const int m = n / 2, total = n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int e = i & 3;
    const int c = (i >> 2) % m;
    const int rest = (i >> 2) / m;   // (js * 4 + part) * 4 + kg
    const int kg = rest & 3, part = (rest >> 2) & 3, js = rest >> 4;
    const int k = js * TC_KB + kg * 4 + e;
    const long long kc = ((long long)k * c) % n;
    double sv, cv;
    sincospi(2.0 * (double)kc / (double)n, &sv, &cv);
    const double v = part < 2 ? cv : sv;
    const uint32_t h = tf32_bits((float)v);
    img[i] = (part & 1) == 0 ? h : tf32_bits((float)(v - (double)__uint_as_float(h)));
  }
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// 3-D map over the rows of X: (4 floats, M rows, n / 4 K-groups), strides
// (n * 4, 16) bytes, box (4, 128, TC_KB / 4); rows past M read as zero
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

bool encode_xmap(CUtensorMap* m, const float* X, int M, int n) {
  const auto encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[3] = {4, (cuuint64_t)M, (cuuint64_t)(n / 4)};
  const cuuint64_t strides[2] = {(cuuint64_t)n * 4, 16};
  const cuuint32_t box[3] = {4, TC_M, TC_KB / 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the same over bfloat16 rows: (8 values, M rows, n / 8 K-groups), strides
// (n * 2, 16) bytes, box (8, 128, TC_KB / 8)
bool encode_xmap_bf16(CUtensorMap* m, const void* X, int M, int n) {
  const auto encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[3] = {8, (cuuint64_t)M, (cuuint64_t)(n / 8)};
  const cuuint64_t strides[2] = {(cuuint64_t)n * 2, 16};
  const cuuint32_t box[3] = {8, TC_M, TC_KB / 8};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(X), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// persistent grids: one CTA per SM, leaving `reserved` SMs to a concurrent kernel
int persistent_grid(int ntiles, int reserved) {
  int n = sm_count() - reserved;
  if (n < sm_count() / 2) n = sm_count() / 2;
  return ntiles < n ? ntiles : n;
}

template <int N>
bool launch_direct(const float* X, const direct::DArgs& g, cudaStream_t s, int reserved) {
  CUtensorMap m;
  if (!encode_xmap(&m, X, g.M, N)) return false;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int grid = persistent_grid(ntiles, reserved);
  direct::k_gemm_tc_direct<N><<<grid, direct::D_THREADS, direct::DCfg<N>::SMEM, s>>>(g, m);
  return true;
}

template <int N, int SPLIT>
bool launch_tc(const float* X, const TcArgs& g, cudaStream_t s, int reserved) {
  CUtensorMap m;
  if (!encode_xmap(&m, X, g.M, N)) return false;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int grid = persistent_grid(ntiles, reserved);
  k_gemm_tc_tf32x3<N, SPLIT><<<grid, TC_THREADS, TcCfg<N, SPLIT>::SMEM, s>>>(g, m);
  return true;
}

bool launch_tc_bf16(const void* X, const b16::Args& g, cudaStream_t s, int reserved) {
  CUtensorMap m;
  if (!encode_xmap_bf16(&m, X, g.M, b16::N)) return false;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int grid = persistent_grid(ntiles, reserved);
  b16::k_gemm_tc_bf16<<<grid, TC_THREADS, b16::SMEM, s>>>(g, m);
  return true;
}

}  // namespace

size_t tc_bf16_image_bytes() { return b16::IMG; }

bool tc_bf16_available(const void* X, int planes) {
  CUtensorMap m;
  return planes > 0 && encode_xmap_bf16(&m, X, planes * b16::N, b16::N);
}

void tc_pack_hartley_bf16(unsigned char* img, cudaStream_t s) {
  b16::k_pack<<<(2 * b16::MH * b16::MH + 255) / 256, 256, 0, s>>>(reinterpret_cast<uint16_t*>(img));
}

// out = (X H)^T for each 256 x 256 plane of X, X and out bfloat16 (16-byte
// aligned, distinct), H the 256-point Hartley matrix as the bfloat16 image of
// tc_pack_hartley_bf16 (resident in shared memory), FP32 accumulation.
// Returns false (nothing launched) when the tensor map cannot be encoded.
bool tc_rows_times_h_bf16(const void* X, const unsigned char* img, void* out, int planes, int* error,
                          cudaStream_t s, int sm_reserved) {
  if (planes <= 0) return true;
  const b16::Args g{img, reinterpret_cast<__nv_bfloat16*>(out), planes * b16::N, error};
  return launch_tc_bf16(X, g, s, sm_reserved);
}

bool tc_supported(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }

// image bytes: the even/odd cos / sin image at 256 (4 n^2), the direct H
// image below (8 n^2)
size_t tc_h_image_bytes(int n) {
  if (!tc_supported(n)) return 0;
  return (size_t)(n == 256 ? 1 : 2) * n * n * sizeof(float);
}

void tc_pack_hartley(int n, unsigned char* img, cudaStream_t s) {
  if (!tc_supported(n)) return;
  if (n == 256) {
    k_pack_hartley<<<(n * n + 255) / 256, 256, 0, s>>>(n, reinterpret_cast<uint32_t*>(img));
  } else {
    direct::k_pack_direct<<<(2 * n * n + 255) / 256, 256, 0, s>>>(n, reinterpret_cast<uint32_t*>(img));
  }
}

// out = (X H)^T for each of the `planes` n x n planes of X (rows of n
// contiguous values), n = 32, 64, 128 or 256, H the n-point Hartley matrix
// given by its pre-split image (tc_pack_hartley): the even/odd form at 256,
// the direct form below; X, out 16-byte aligned, out distinct from X. error:
// device flag that receives ERR_TIMEOUT if a bounded wait runs out. single:
// the single TF32 product at 256 (whichever solve of the refinement may be
// coarse); the split products otherwise. sm_reserved: SMs held by a concurrent kernel, which
// the persistent grid leaves free. Returns false (nothing launched) for other
// n or when the tensor map cannot be encoded.
bool tc_rows_times_h_t(const float* X, const unsigned char* img, float* out, int planes, int n, int* error,
                       cudaStream_t s, bool single, int sm_reserved) {
  if (planes <= 0) return tc_supported(n);
  if (n == 256) {
    TcArgs g{img, out, planes * n, error};
    return single ? launch_tc<256, 1>(X, g, s, sm_reserved) : launch_tc<256, 3>(X, g, s, sm_reserved);
  }
  direct::DArgs d{img, out, planes * n, error};
  switch (n) {
    case 32: return launch_direct<32>(X, d, s, sm_reserved);
    case 64: return launch_direct<64>(X, d, s, sm_reserved);
    case 128: return launch_direct<128>(X, d, s, sm_reserved);
    default: return false;
  }
}

void tc_gemm_set_attributes() {
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<256, 3>::SMEM);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<256, 1>::SMEM);
  cudaFuncSetAttribute(direct::k_gemm_tc_direct<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)direct::DCfg<32>::SMEM);
  cudaFuncSetAttribute(direct::k_gemm_tc_direct<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)direct::DCfg<64>::SMEM);
  cudaFuncSetAttribute(direct::k_gemm_tc_direct<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)direct::DCfg<128>::SMEM);
  cudaFuncSetAttribute(b16::k_gemm_tc_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b16::SMEM);
}

}  // namespace ibm
