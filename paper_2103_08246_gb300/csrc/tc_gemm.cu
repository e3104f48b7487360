// Split-TF32 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a) for
// the Hartley transforms of the mixed-precision pressure solve: for every
// n x n plane X (n = 32, 64, 128 or 256; rows of n contiguous values) it
// computes
//   out = (X H)^T,   H = H^T the n-point Hartley matrix,
// with FP32 operands rounded as a ~ a_hi + a_lo, a_hi = tf32(a),
// a_lo = tf32(a - a_hi) (round to nearest, ties away), and
// a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in FP32 in tensor memory.
// Applied twice, ((X H)^T H)^T = H X H: the 2-D transform of the plane, with
// both GEMMs reading K-major rows.
//
// Persistent and warp-specialised, one CTA per SM, tiles of 128 rows (of one
// or several planes) x n columns, K in blocks of 16 through a four-stage
// shared-memory ring:
//  * warp 0 (one thread) fills a stage with one tensor-map copy of the A
//    block, which lands directly in the K-major core-matrix layout (box of
//    4 floats x 128 rows x 4 K-groups: [K-group][row][16 bytes]), and one
//    bulk copy of the block's slice of the pre-split H image (hi and lo
//    tiles in the same layout, built once by tc_pack_h);
//  * warps 2-7 split the A block in place: a_hi over the raw values, a_lo
//    into the stage's second A tile;
//  * warp 1 (one thread) issues the 2 x 3 tcgen05.mma (M = 128, N = n,
//    K = 8) of the block into one of two tensor-memory accumulators and
//    commits them to the stage's "empty" barrier (and, after the tile's last
//    block, to the accumulator's "full" barrier);
//  * warps 8-15 read the other accumulator back with tcgen05.ld (warp w its
//    lane quarter w % 4, half of the columns) and store it transposed into
//    the plane: for every column the warp's 32 rows are 32 consecutive
//    floats. Rows past the last plane load zeros (the tensor map's
//    out-of-range fill) and store nothing.
// Every mbarrier wait is bounded; on expiry the waiting thread records it
// and carries on, the kernel sets the error flag, waits (bounded) for its own
// tensor-core work, releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "solver.h"
#include "tcgen05.cuh"

namespace ibm {

namespace {

constexpr int TC_M = 128, TC_KB = 16, TC_STAGES = 4;
constexpr int TC_THREADS = 512;                    // 16 warps
constexpr int TC_CONV_WARPS = 6, TC_EPI_WARPS = 8;
constexpr uint32_t A_TILE = TC_M * TC_KB * 4;      // bytes of one A part (hi or lo)
constexpr uint32_t A_LBO = TC_M * 16;              // K-adjacent core matrices of A
template <int N>
struct TcCfg {
  static constexpr uint32_t B_TILE = (uint32_t)N * TC_KB * 4;
  static constexpr uint32_t B_LBO = (uint32_t)N * 16;
  static constexpr uint32_t STAGE = 2 * A_TILE + 2 * B_TILE;   // A_hi, A_lo, B_hi, B_lo
  static constexpr uint32_t SMEM = TC_STAGES * STAGE;
  static constexpr uint32_t TMEM_COLS = 2 * N;                 // two accumulators
  static constexpr int NKB = N / TC_KB;
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

struct TcArgs {
  const unsigned char* himg;   // pre-split H (tc_pack_h)
  float* out;                  // per plane: out[c][r] = sum_k X[r][k] H[k][c]
  int M;                       // rows of X (planes x n)
  int* error;
};

template <int N>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc_tf32x3(TcArgs g, const __grid_constant__ CUtensorMap xmap) {
  using C = TcCfg<N>;
  constexpr uint32_t A_TX = A_TILE, B_TX = 2 * C::B_TILE;
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t full[TC_STAGES], conv[TC_STAGES], empty[TC_STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * C::NKB;
  const uint32_t sbase = smem_u32(tsm);

  if (warp == 0) tc_alloc(&tmem_slot, C::TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], TC_CONV_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TC_EPI_WARPS);
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
        const int s = j % TC_STAGES;
        if (j >= TC_STAGES) ok = mbar_wait(&empty[s], (uint32_t)(j / TC_STAGES - 1) & 1u) && ok;
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
        const int s = j % TC_STAGES;
        const int lt = j / C::NKB, kb = j % C::NKB;
        // the accumulator's previous tile (lt - 2) must have been read out
        if (kb == 0 && lt >= 2) ok = mbar_wait(&tempty[lt & 1], (uint32_t)((lt - 2) / 2) & 1u) && ok;
        ok = mbar_wait(&conv[s], (uint32_t)(j / TC_STAGES) & 1u) && ok;
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
  } else if (warp < 2 + TC_CONV_WARPS) {
    // split: 16-byte chunks of the A block, a_hi in place, a_lo to the second tile
    const int ct = tid - 64;
    constexpr int CHUNKS = A_TILE / 16;
    for (int j = 0; j < total; ++j) {
      const int s = j % TC_STAGES;
      ok = mbar_wait(&full[s], (uint32_t)(j / TC_STAGES) & 1u) && ok;
      uint4* hi = reinterpret_cast<uint4*>(tsm + (size_t)s * C::STAGE);
      uint4* lo = reinterpret_cast<uint4*>(tsm + (size_t)s * C::STAGE + A_TILE);
      for (int q = ct; q < CHUNKS; q += 32 * TC_CONV_WARPS) {
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
// [K-group][n][4 floats] (element (c, k) = H[k][c]); one thread per value
__global__ void k_pack_h(const float* __restrict__ H, int n, uint32_t* __restrict__ img) {
  const int total = 2 * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int e = i & 3;
    const int c = (i >> 2) % n;
    const int rest = (i >> 2) / n;              // (kb * 2 + part) * (TC_KB / 4) + kg
    const int kg = rest % (TC_KB / 4);
    const int part = (rest / (TC_KB / 4)) & 1;
    const int kb = rest / (2 * (TC_KB / 4));
    const int k = kb * TC_KB + kg * 4 + e;
    const float x = H[(size_t)k * n + c];
    const uint32_t h = tf32_bits(x);
    img[i] = part == 0 ? h : tf32_bits(x - __uint_as_float(h));
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
bool encode_xmap(CUtensorMap* m, const float* X, int M, int n) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {4, (cuuint64_t)M, (cuuint64_t)(n / 4)};
  const cuuint64_t strides[2] = {(cuuint64_t)n * 4, 16};
  const cuuint32_t box[3] = {4, TC_M, TC_KB / 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
bool launch_tc(const float* X, const TcArgs& g, cudaStream_t s) {
  CUtensorMap m;
  if (!encode_xmap(&m, X, g.M, N)) return false;
  const int ntiles = (g.M + TC_M - 1) / TC_M;
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  k_gemm_tc_tf32x3<N><<<grid, TC_THREADS, TcCfg<N>::SMEM, s>>>(g, m);
  return true;
}

}  // namespace

bool tc_supported(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }

size_t tc_h_image_bytes(int n) { return tc_supported(n) ? (size_t)2 * n * n * sizeof(float) : 0; }

void tc_pack_h(const float* H, int n, unsigned char* img, cudaStream_t s) {
  if (!tc_supported(n)) return;
  const int total = 2 * n * n;
  k_pack_h<<<(total + 255) / 256, 256, 0, s>>>(H, n, reinterpret_cast<uint32_t*>(img));
}

// out = (X H)^T for each of the `planes` n x n planes of X (rows of n
// contiguous values), n = 32, 64, 128 or 256, H given by its pre-split image
// (tc_pack_h); X, out 16-byte aligned, out distinct from X. error: device
// flag that receives ERR_TIMEOUT if a bounded wait runs out. Returns false
// (nothing launched) for other n or when the tensor map cannot be encoded.
bool tc_rows_times_h_t(const float* X, const unsigned char* himg, float* out, int planes, int n, int* error,
                       cudaStream_t s) {
  if (planes <= 0) return tc_supported(n);
  TcArgs g{himg, out, planes * n, error};
  switch (n) {
    case 32: return launch_tc<32>(X, g, s);
    case 64: return launch_tc<64>(X, g, s);
    case 128: return launch_tc<128>(X, g, s);
    case 256: return launch_tc<256>(X, g, s);
    default: return false;
  }
}

void tc_gemm_set_attributes() {
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<32>::SMEM);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<64>::SMEM);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<128>::SMEM);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<256>::SMEM);
}

}  // namespace ibm
