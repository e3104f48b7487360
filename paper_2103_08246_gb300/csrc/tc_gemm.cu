// Split-TF32 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a) for
// the Hartley transforms of the mixed-precision pressure solve: for every
// n x n plane X (n = 32, 64, 128 or 256; rows of n contiguous values) it
// computes
//   out = (X H)^T,   H = H^T the n-point Hartley matrix,
// with FP32 operands rounded as a ~ a_hi + a_lo, a_hi = tf32(a),
// a_lo = tf32(a - a_hi), and a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated in
// FP32 in tensor memory. Applied twice, ((X H)^T H)^T = H X H: the 2-D
// transform of the plane, with both GEMMs reading K-major rows.
//
// One CTA (4 warps) computes 128 rows (of one or several planes) x n columns
// of X H over K in blocks of 32:
//  * all threads load the next K block (A: 128 x 32, B: n x 32) from global
//    memory into registers while the tensor core works on the current one,
//    split it into hi / lo parts and store both into shared memory in the
//    K-major "core matrix" layout (8 rows x 16 bytes per 128-byte core
//    matrix; core matrices adjacent in K are 128 bytes apart, adjacent in
//    M / N 1024 bytes apart);
//  * one thread issues the 4 x 3 tcgen05.mma (M = 128, N = n, K = 8 each)
//    of the block and commits them to the stage's mbarrier, which the
//    loaders wait on before they overwrite that stage;
//  * the accumulator (128 lanes x n FP32 columns of tensor memory) is read
//    back with tcgen05.ld, each warp its 32 lanes (rows, all in one plane as
//    32 divides n), and stored transposed into the plane: for every column
//    the warp's 32 rows are 32 consecutive floats. Rows past the last plane
//    (when 128 does not divide planes x n) load zeros and store nothing.
// Every mbarrier wait is bounded; on expiry the kernel sets the error flag,
// still waits (bounded) for its own tensor-core work, releases its tensor
// memory and returns.
#include <cstdint>

#include "solver.h"
#include "tcgen05.cuh"

namespace ibm {

namespace {

constexpr int TC_M = 128, TC_KB = 32;
constexpr int TC_THREADS = 128;
constexpr uint32_t A_TILE = TC_M * TC_KB * 4;   // bytes of one A part (hi or lo)
template <int N>
struct TcCfg {
  static constexpr uint32_t B_TILE = N * TC_KB * 4;
  static constexpr uint32_t STAGE = 2 * A_TILE + 2 * B_TILE;   // A_hi, A_lo, B_hi, B_lo (one stage)
  static constexpr uint32_t TMEM_COLS = N < 32 ? 32 : N;
};

// byte offset of element (row, k) of a K-major tile with TC_KB columns
__device__ inline uint32_t kmajor_off(int row, int k) {
  return (uint32_t)(((row >> 3) * (TC_KB / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

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

// K-major operand tiles: K-groups 128 bytes apart, 8-row groups 1024 bytes apart
__device__ inline uint64_t kdesc(uint32_t saddr) { return tc_desc(saddr, 128, 1024); }

__device__ inline void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

struct TcArgs {
  const float* X;   // rows of n values (M rows, planes of n rows)
  const float* H;   // n x n, symmetric
  float* out;       // per plane: out[c][r] = sum_k X[r][k] H[k][c]
  int M;
  int* error;
};

template <int N>
__global__ void __launch_bounds__(TC_THREADS, 2) k_gemm_tc_tf32x3(TcArgs g) {
  using C = TcCfg<N>;
  constexpr uint32_t B_TILE = C::B_TILE, STAGE = C::STAGE;
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ uint64_t done[1];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * TC_M;
  const float* A = g.X;
  const float* B = g.H;
  constexpr int LD = N;
  const uint32_t sbase = smem_u32(tsm);

  if (warp == 0) {
    tc_alloc(&tmem_base, C::TMEM_COLS);
  }
  if (tid == 0) {
    mbar_init(&done[0], 1);
    fence_mbar_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // register staging of one K block: A 8 float4, B N / 16 float4 per thread.
  // float4 number e holds row (e >> 6) * 8 + (e & 7), columns 4 ((e >> 3) & 7)
  // .. + 3: the 8 lanes of a shared-store phase fill one 128-byte core matrix.
  auto row_of = [](int e) { return (e >> 6) * 8 + (e & 7); };
  auto col_of = [](int e) { return ((e >> 3) & 7) * 4; };
  constexpr int NB4 = N / 16;
  float4 ra[8], rb[NB4];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + t * TC_THREADS;   // 1024 float4 of A (128 rows x 32)
      const int m = m0 + row_of(e);
      ra[t] = m < g.M ? *reinterpret_cast<const float4*>(A + (size_t)m * LD + k0 + col_of(e))
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < NB4; ++t) {
      const int e = tid + t * TC_THREADS;   // N * 8 float4 of B (N rows x 32)
      rb[t] = *reinterpret_cast<const float4*>(B + (size_t)row_of(e) * LD + k0 + col_of(e));
    }
  };
  auto split_store = [&](unsigned char* hi_tile, unsigned char* lo_tile, int row, int c4,
                         const float4& v) {
    const float x[4] = {v.x, v.y, v.z, v.w};
    uint4 hi, lo;
    uint32_t* ph = &hi.x;
    uint32_t* pl = &lo.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ph[q] = tf32_bits(x[q]);
      pl[q] = tf32_bits(x[q] - __uint_as_float(ph[q]));
    }
    const uint32_t off = kmajor_off(row, c4);
    *reinterpret_cast<uint4*>(hi_tile + off) = hi;
    *reinterpret_cast<uint4*>(lo_tile + off) = lo;
  };
  auto put = [&](unsigned char* st) {
    unsigned char* ah = st;
    unsigned char* al = st + A_TILE;
    unsigned char* bh = st + 2 * A_TILE;
    unsigned char* bl = st + 2 * A_TILE + B_TILE;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + t * TC_THREADS;
      split_store(ah, al, row_of(e), col_of(e), ra[t]);
    }
#pragma unroll
    for (int t = 0; t < NB4; ++t) {
      const int e = tid + t * TC_THREADS;
      split_store(bh, bl, row_of(e), col_of(e), rb[t]);
    }
    // make the generic-proxy stores visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  constexpr uint32_t idesc = tc_idesc(N);
  auto issue = [&](int s, bool first) {
    const uint32_t st = sbase + (uint32_t)s * STAGE;
    const uint32_t ah = st, al = st + A_TILE, bh = st + 2 * A_TILE, bl = st + 2 * A_TILE + B_TILE;
#pragma unroll
    for (int kk = 0; kk < TC_KB / 8; ++kk) {
      const uint32_t ko = (uint32_t)kk * 256;   // two core matrices (K = 8) per step
      tc_mma(tmem, kdesc(ah + ko), kdesc(bh + ko), idesc, (first && kk == 0) ? 0u : 1u);
      tc_mma(tmem, kdesc(ah + ko), kdesc(bl + ko), idesc, 1u);
      tc_mma(tmem, kdesc(al + ko), kdesc(bh + ko), idesc, 1u);
    }
    tc_commit_to(&done[s]);
  };

  const int nk = N / TC_KB;
  bool ok = true;
  load(0);
  for (int kb = 0; kb < nk; ++kb) {
    // the stage's previous MMAs (block kb - 1) must be done before it is overwritten
    if (kb > 0) ok = mbar_wait(&done[0], (uint32_t)(kb - 1) & 1u) && ok;
    put(tsm);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(0, kb == 0);
    }
    if (kb + 1 < nk) load((kb + 1) * TC_KB);
  }
  // all MMAs complete: the last commit
  ok = mbar_wait(&done[0], (uint32_t)(nk - 1) & 1u) && ok;
  // one decision for the whole CTA: the tensor-memory loads below are warp-collective
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok && tid == 0) atomicOr(g.error, ERR_TIMEOUT);
  if (ok) {
    // warp w owns accumulator lanes (rows) 32 w .. 32 w + 31; row m = plane * N + r
    const int m = m0 + warp * 32 + (tid & 31);
    float* plane = g.out + (size_t)(m / N) * N * N + (m % N);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tc_ld_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < g.M) {
#pragma unroll
        for (int q = 0; q < 32; ++q) plane[(size_t)(c0 + q) * N] = v[q];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    tc_dealloc(tmem, C::TMEM_COLS);
}

template <int N>
void launch_tc(const TcArgs& g, cudaStream_t s) {
  k_gemm_tc_tf32x3<N><<<(g.M + TC_M - 1) / TC_M, TC_THREADS, TcCfg<N>::STAGE, s>>>(g);
}

}  // namespace

// out = (X H)^T for each of the `planes` n x n planes of X (rows of n
// contiguous values), n = 32, 64, 128 or 256; X, H, out 16-byte aligned, out
// distinct from X. error: device flag that receives ERR_TIMEOUT if a bounded
// wait runs out. Returns false for other n (nothing launched).
bool tc_rows_times_h_t(const float* X, const float* H, float* out, int planes, int n, int* error,
                       cudaStream_t s) {
  TcArgs g{X, H, out, planes * n, error};
  switch (n) {
    case 32: launch_tc<32>(g, s); return true;
    case 64: launch_tc<64>(g, s); return true;
    case 128: launch_tc<128>(g, s); return true;
    case 256: launch_tc<256>(g, s); return true;
    default: return false;
  }
}

void tc_gemm_set_attributes() {
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<32>::STAGE);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<64>::STAGE);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<128>::STAGE);
  cudaFuncSetAttribute(k_gemm_tc_tf32x3<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<256>::STAGE);
}

}  // namespace ibm
