// Mixed-precision pressure solve (FP32 fields): a predictor solve, an
// extended-precision (double-single, FP64-class) evaluation of the residual
// r = D - L_h phi and one refinement sweep (a correction solve applied to r,
// phi += delta). The transverse transforms of the correction (and of the
// predictor where no FFT serves the plane size) are dense contractions with
// the Hartley matrices H_n[j][k] = cas(2 pi j k / n) (Sec. II.B projection
// step), run on tensor cores as TF32 GEMMs with FP32 accumulation, single
// (a_hi b_hi) or split,
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,  a_hi = tf32(a), a_lo = tf32(a - a_hi).
//
// 2-D transform of every x plane X (ny x nz, z contiguous): H_y X H_z, as
// two GEMMs: rows (all planes at once) times H_z, then H_y times each plane.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "solver.h"

namespace ibm {

constexpr int GBM = 128, GBN = 128, GBK = 32;
constexpr int AS_LD = GBK + 4;    // shared row strides: conflict-free fragment reads
constexpr int BS_LD = GBN + 8;

struct GemmArgs {
  const float* A;
  const float* B;
  float* C;
  int M, N, K;
  int lda, ldb, ldc;
  long long sA, sB, sC;   // batch strides (elements)
};

__device__ inline uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ inline void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[b] = A[b] (M x K) * B[b] (K x N), row-major, batched over blockIdx.z.
// 8 warps: 2 along M (64 rows each) x 4 along N (32 columns each).
__global__ void __launch_bounds__(256) k_gemm_tf32x3(GemmArgs g) {
  extern __shared__ __align__(16) float gsm[];
  float* As = gsm;                         // [2][GBM][AS_LD]
  float* Bs = gsm + 2 * GBM * AS_LD;       // [2][GBK][BS_LD]
  const int bz = blockIdx.z;
  const float* A = g.A + bz * g.sA;
  const float* B = g.B + bz * g.sB;
  float* C = g.C + bz * g.sC;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  const bool full = (m0 + GBM <= g.M) && (n0 + GBN <= g.N) && (g.K % GBK == 0) &&
                    (g.lda % 4 == 0) && (g.ldb % 4 == 0);
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][b][q] = 0.f;

  float4 ra[4], rb[4];
  auto load_regs = [&](int k0) {
    if (full) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = tid + t * 256;            // 1024 float4 of A (128 x 32)
        const int r = e >> 3, c4 = (e & 7) * 4;
        ra[t] = *reinterpret_cast<const float4*>(A + (size_t)(m0 + r) * g.lda + k0 + c4);
        const int rr = e >> 5, cc = (e & 31) * 4;  // 1024 float4 of B (32 x 128)
        rb[t] = *reinterpret_cast<const float4*>(B + (size_t)(k0 + rr) * g.ldb + n0 + cc);
      }
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = tid + t * 256;
        const int r = e >> 3, c4 = (e & 7) * 4;
        float v[4];
        for (int q = 0; q < 4; ++q) {
          const int m = m0 + r, k = k0 + c4 + q;
          v[q] = (m < g.M && k < g.K) ? A[(size_t)m * g.lda + k] : 0.f;
        }
        ra[t] = make_float4(v[0], v[1], v[2], v[3]);
        const int rr = e >> 5, cc = (e & 31) * 4;
        for (int q = 0; q < 4; ++q) {
          const int k = k0 + rr, n = n0 + cc + q;
          v[q] = (k < g.K && n < g.N) ? B[(size_t)k * g.ldb + n] : 0.f;
        }
        rb[t] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  };
  auto store_regs = [&](int buf) {
    float* as = As + buf * GBM * AS_LD;
    float* bs = Bs + buf * GBK * BS_LD;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;
      const int r = e >> 3, c4 = (e & 7) * 4;
      float* pa = as + r * AS_LD + c4;
      pa[0] = ra[t].x;
      pa[1] = ra[t].y;
      pa[2] = ra[t].z;
      pa[3] = ra[t].w;
      const int rr = e >> 5, cc = (e & 31) * 4;
      float* pb = bs + rr * BS_LD + cc;
      pb[0] = rb[t].x;
      pb[1] = rb[t].y;
      pb[2] = rb[t].z;
      pb[3] = rb[t].w;
    }
  };
  const int nk = (g.K + GBK - 1) / GBK;
  load_regs(0);
  store_regs(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) load_regs((kt + 1) * GBK);
    const float* as = As + buf * GBM * AS_LD;
    const float* bs = Bs + buf * GBK * BS_LD;
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 8) {
      uint32_t ahi[4][4], alo[4][4], bhi[4][2], blo[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const float* p = as + (wm + mt * 16 + gid) * AS_LD + kk + tig;
        const float x[4] = {p[0], p[8 * AS_LD], p[4], p[8 * AS_LD + 4]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ahi[mt][q] = tf32_of(x[q]);
          alo[mt][q] = tf32_of(x[q] - __uint_as_float(ahi[mt][q]));
        }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const float* p = bs + (kk + tig) * BS_LD + wn + nt * 8 + gid;
        const float x[2] = {p[0], p[4 * BS_LD]};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          bhi[nt][q] = tf32_of(x[q]);
          blo[nt][q] = tf32_of(x[q] - __uint_as_float(bhi[nt][q]));
        }
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_tf32(acc[mt][nt], alo[mt], bhi[nt]);
          mma_tf32(acc[mt][nt], ahi[mt], blo[nt]);
          mma_tf32(acc[mt][nt], ahi[mt], bhi[nt]);
        }
    }
    if (kt + 1 < nk) {
      __syncthreads();
      store_regs(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int r = m0 + wm + mt * 16 + gid;
      const int cidx = n0 + wn + nt * 8 + 2 * tig;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = r + 8 * h;
        if (rr >= g.M) continue;
        if (cidx < g.N) C[(size_t)rr * g.ldc + cidx] = acc[mt][nt][2 * h];
        if (cidx + 1 < g.N) C[(size_t)rr * g.ldc + cidx + 1] = acc[mt][nt][2 * h + 1];
      }
    }
}

// Residual r = D - L_h phi (Neumann x ends, periodic y, z) of FP32 D and phi,
// stored in FP32, evaluated in double-single arithmetic: every sum and product
// is an error-free transformation on the FP32 pipe (Knuth's TwoSum; the
// FMA-based exact product), so the seven-point sum is carried as an
// unevaluated pair hi + lo with a relative error of about 2^-47 of the
// stencil's terms, well below the FP32 rounding of the stored residual. Same
// accuracy class as an FP64 evaluation, without the FP64 pipe (2 instructions
// per clock per SM on this part, against 128 FP32). The _rn intrinsics keep
// the compiler from contracting products into the sums.
struct DS {
  float hi, lo;
};

__device__ inline DS two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// residual of one cell from its value, six neighbours and D, with
// ih2 = ih2_hi + ih2_lo the host-split 1 / h^2. POW2: 1 / h^2 is a power of
// two (ih2_lo = 0), so S ih2 is exact as the pair (S.hi ih2, S.lo ih2) and
// the product's error terms vanish (the same values with fewer operations)
template <bool POW2>
__device__ inline float residual_ds(float pc, float pxm, float pxp, float pym, float pyp, float pzm, float pzp,
                                    float D, float ih2_hi, float ih2_lo) {
  // S = sum of the six neighbours - 6 pc, as hi + lo
  const DS s1 = two_sum(pxm, pxp), s2 = two_sum(pym, pyp), s3 = two_sum(pzm, pzp);
  const DS s4 = two_sum(s1.hi, s2.hi), s5 = two_sum(s4.hi, s3.hi);
  const float p6 = __fmul_rn(6.0f, pc);
  const float q6 = __fmaf_rn(6.0f, pc, -p6);   // 6 pc = p6 + q6 exactly
  const DS s6 = two_sum(s5.hi, -p6);
  const float lo = __fsub_rn(
      __fadd_rn(__fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(s3.lo, s4.lo)), __fadd_rn(s5.lo, s6.lo)), q6);
  const DS S = two_sum(s6.hi, lo);
  // lap = S ih2 (exact leading product plus the cross terms)
  DS lap;
  if constexpr (POW2) {
    lap = {__fmul_rn(S.hi, ih2_hi), __fmul_rn(S.lo, ih2_hi)};
  } else {
    const float ph = __fmul_rn(S.hi, ih2_hi);
    const float pe = __fadd_rn(__fmaf_rn(S.hi, ih2_hi, -ph),
                               __fadd_rn(__fmul_rn(S.hi, ih2_lo), __fmul_rn(S.lo, ih2_hi)));
    lap = two_sum(ph, pe);
  }
  // r = D - lap
  const DS t = two_sum(D, -lap.hi);
  return __fadd_rn(t.hi, __fsub_rn(t.lo, lap.lo));
}

// four consecutive z cells per thread (nz is a power of two >= 4): 16-byte loads of
// the cell run and of its x and y neighbours, the two z neighbours past the
// run's ends as single loads; grid (z runs, y rows, x planes)
template <class R, bool POW2>
__global__ void k_residual_ds4(int nx, int ny, int nz, float ih2_hi, float ih2_lo, const float* __restrict__ D,
                               const float* __restrict__ phi, R* __restrict__ r) {
  const int k0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (k0 >= nz) return;
  const int j = blockIdx.y, i = blockIdx.z;
  const size_t P = (size_t)ny * nz;
  const size_t row = (size_t)i * P + (size_t)j * nz;
  const size_t id = row + k0;
  const float4 c4 = *reinterpret_cast<const float4*>(phi + id);
  const float4 xm = i > 0 ? *reinterpret_cast<const float4*>(phi + id - P) : c4;
  const float4 xp = i < nx - 1 ? *reinterpret_cast<const float4*>(phi + id + P) : c4;
  const size_t rm = (size_t)i * P + (size_t)(j == 0 ? ny - 1 : j - 1) * nz + k0;
  const size_t rp = (size_t)i * P + (size_t)(j == ny - 1 ? 0 : j + 1) * nz + k0;
  const float4 ym = *reinterpret_cast<const float4*>(phi + rm);
  const float4 yp = *reinterpret_cast<const float4*>(phi + rp);
  const float zl = phi[row + (k0 == 0 ? nz - 1 : k0 - 1)];
  const float zr = phi[row + (k0 + 4 == nz ? 0 : k0 + 4)];
  const float4 d4 = *reinterpret_cast<const float4*>(D + id);
  float4 o;
  o.x = residual_ds<POW2>(c4.x, xm.x, xp.x, ym.x, yp.x, zl, c4.y, d4.x, ih2_hi, ih2_lo);
  o.y = residual_ds<POW2>(c4.y, xm.y, xp.y, ym.y, yp.y, c4.x, c4.z, d4.y, ih2_hi, ih2_lo);
  o.z = residual_ds<POW2>(c4.z, xm.z, xp.z, ym.z, yp.z, c4.y, c4.w, d4.z, ih2_hi, ih2_lo);
  o.w = residual_ds<POW2>(c4.w, xm.w, xp.w, ym.w, yp.w, c4.z, zr, d4.w, ih2_hi, ih2_lo);
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(r + id) = o;
  } else {   // bfloat16: the correction's input
    const __nv_bfloat162 a = __floats2bfloat162_rn(o.x, o.y), b = __floats2bfloat162_rn(o.z, o.w);
    *reinterpret_cast<uint2*>(r + id) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
}

// the residual kernel for this 1 / h^2 (exact pair products when it is a power of two)
template <class R>
static void launch_residual(const Consts& c, const float* D, const float* x0, R* r, cudaStream_t s) {
  const double ih2 = c.inv_h * c.inv_h;
  const float ih2_hi = (float)ih2, ih2_lo = (float)(ih2 - (double)ih2_hi);
  int e = 0;
  const bool pow2 = ih2_lo == 0.f && std::frexp((double)ih2_hi, &e) == 0.5;
  const dim3 grid((c.nz / 4 + 63) / 64, c.ny, c.nx);
  if (pow2)
    k_residual_ds4<R, true><<<grid, 64, 0, s>>>(c.nx, c.ny, c.nz, ih2_hi, ih2_lo, D, x0, r);
  else
    k_residual_ds4<R, false><<<grid, 64, 0, s>>>(c.nx, c.ny, c.nz, ih2_hi, ih2_lo, D, x0, r);
}

static void gemm(const GemmArgs& g, int batch, cudaStream_t s) {
  const size_t sh = (size_t)(2 * GBM * AS_LD + 2 * GBK * BS_LD) * sizeof(float);
  k_gemm_tf32x3<<<dim3((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, batch), 256, sh, s>>>(g);
}

// 2-D Hartley transform of every x plane: out = H_y in H_z (tmp: scratch).
// Square planes of 32, 64, 128 or 256 run on the tcgen05 tensor cores as two
// passes out = ((in H)^T H)^T; other shapes on the mma.sync kernel above.
// The two tensor-core passes differ only in their (16-byte aligned) input,
// so the second launches wherever the first did.
struct Hartley {
  const float* y;
  const float* z;
  const unsigned char* y_img;
  const unsigned char* z_img;
};

static void transform2d(const Consts& c, const Hartley& H, const float* in, float* tmp, float* out, int* error,
                        cudaStream_t s, bool single = false) {
  if (c.ny == c.nz && H.z_img &&
      tc_rows_times_h_t(in, H.z_img, tmp, c.nx, c.nz, error, s, single, c.sm_reserved)) {
    tc_rows_times_h_t(tmp, H.y_img, out, c.nx, c.ny, error, s, single, c.sm_reserved);
    return;
  }
  const long long P = (long long)c.ny * c.nz;
  GemmArgs a{in, H.z, tmp, c.nx * c.ny, c.nz, c.nz, c.nz, c.nz, c.nz, 0, 0, 0};
  gemm(a, 1, s);
  GemmArgs b{H.y, tmp, out, c.ny, c.nz, c.ny, c.ny, c.nz, c.nz, 0, P, P};
  gemm(b, c.nx, s);
}

// e[1] + e[2] <- solution of L_h phi = D (D in f.phi on entry), mixed precision
// with one refinement sweep on the extended-precision residual; the
// projection sums the two parts as it reads them (no separate pass).
// x0 + t1 with t1 = L^-1 (D - L x0) leaves the correction's relative error
// times the predictor's, so one of the two solves may be coarse. At 256 x 256
// planes (c.corr_bf16) the predictor is the FP32 FFT solve (relative error
// near FP32 rounding) and the whole correction is held in bfloat16: the
// residual rounded to bfloat16, the tensor-core transforms on bfloat16
// operands with FP32 accumulation, the Thomas sweeps in FP32 arithmetic on
// bfloat16 storage (relative error about 2^-8 altogether), half the bytes of
// an FP32 correction. Otherwise both solves run on the tensor cores with FP32
// storage, the predictor with the single TF32 product where it exists (256),
// the correction with the split products. Scratch: e[0], e[1], e[2]
// (bfloat16 correction: the first halves of e[0] and e[2]).
void launch_poisson_mixed(const Consts& c, const Fields<float>& f, const float* Hy, const float* Hz,
                          const unsigned char* Hy_img, const unsigned char* Hz_img, const unsigned char* H16_img,
                          cudaStream_t s) {
  const Hartley H{Hy, Hz, Hy_img, Hz_img};
  float* D = f.phi;
  float* t0 = f.e[0];
  float* x0 = f.e[1];
  float* t1 = f.e[2];
  int* err = &f.prm->error;
  if (c.corr_bf16) {
    // predictor: x0 = L^-1 D by the FP32 FFT solve
    launch_dht2d_on(c, f, D, x0, s);
    launch_poisson_x_on(c, f, x0, s);
    launch_dht2d_on(c, f, x0, x0, s);
    // residual (double-single) and correction, in bfloat16
    __nv_bfloat16* r16 = reinterpret_cast<__nv_bfloat16*>(t1);
    __nv_bfloat16* w16 = reinterpret_cast<__nv_bfloat16*>(t0);
    launch_residual(c, D, x0, r16, s);
    tc_rows_times_h_bf16(r16, H16_img, w16, c.nx, err, s, c.sm_reserved);
    tc_rows_times_h_bf16(w16, H16_img, r16, c.nx, err, s, c.sm_reserved);
    launch_poisson_x_bf16(c, f, r16, s);
    tc_rows_times_h_bf16(r16, H16_img, w16, c.nx, err, s, c.sm_reserved);
    tc_rows_times_h_bf16(w16, H16_img, r16, c.nx, err, s, c.sm_reserved);
    return;
  }
  // predictor: x0 = L^-1 D
  transform2d(c, H, D, t0, x0, err, s, true);
  launch_poisson_x_on(c, f, x0, s);
  transform2d(c, H, x0, t0, x0, err, s, true);
  // double-single residual and correction: t1 = L^-1 (D - L x0)
  launch_residual(c, D, x0, t1, s);
  transform2d(c, H, t1, t0, t1, err, s);
  launch_poisson_x_on(c, f, t1, s);
  transform2d(c, H, t1, t0, t1, err, s);
}

// the refinement's residual alone (stage timing): e[2] = D - L_h e[1]
void launch_residual_mixed(const Consts& c, const Fields<float>& f, cudaStream_t s) {
  if (c.corr_bf16)
    launch_residual(c, f.phi, f.e[1], reinterpret_cast<__nv_bfloat16*>(f.e[2]), s);
  else
    launch_residual(c, f.phi, f.e[1], f.e[2], s);
}

void mixed_set_attributes() {
  cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  tc_gemm_set_attributes();
}

// Hartley matrices in FP32 (entries from FP64 cos/sin of 2 pi j k / n, jk mod n)
void hartley_matrix(int n, float* host) {
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      const long long jk = ((long long)j * k) % n;
      const double a = 2.0 * M_PI * (double)jk / n;
      host[(size_t)j * n + k] = (float)(std::cos(a) + std::sin(a));
    }
}

}  // namespace ibm
