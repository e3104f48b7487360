// Fluid kernels of one fractional step (Sec. II.B): per-step parameters,
// explicit right-hand side (AB2 advection, explicit half of Crank--Nicolson,
// pressure gradient), convective outflow (Sec. II.A), the three implicit
// factors of the approximate factorisation, the mass fix and divergence, and
// the projection with the pressure update.
//
// Layout: x slowest, z fastest; u, v, w have nx + 1 planes (u: faces
// 0..nx; v, w: cells 0..nx-1 plus the outflow ghost plane nx), p and phi nx.
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstring>

#include "async_copy.cuh"
#include "solver.h"

namespace ibm {

constexpr int TK = 32;       // threads along z in 3-D kernels
constexpr int TJ = 8;        // threads along y
constexpr int XCHUNK = 8;    // x planes per block in 3-D kernels

// ---------------------------------------------------------------- parameters
// Warm-up of the segmented implicit line solves: the LU recursions of the
// factors (1 - a L_d) forget their start like rho^k, rho = exp(-theta), so a
// segment started H points early is exact to rho^H (below 1e-17 in FP64,
// 1e-9 in FP32).
constexpr int SEG = 32;      // outputs per thread in the implicit line solves
constexpr int HMAX = 24;     // largest warm-up the segments carry
// FP32 runs stop at the warm-up that covers the same diffusion numbers (the
// FP32 tolerance needs about half the planes): smaller shared-memory segments
template <class T> constexpr int hmax_of() { return sizeof(T) == 8 ? HMAX : 13; }

__device__ inline double af_theta(double r) { return 2.0 * asinh(0.5 / sqrt(r)); }

// dt (fixed or CFL), AB2 weights, implicit diffusion number and sub-steps.
// The per-block speed maxima are non-negative doubles (or +inf), whose bit
// patterns order like the values, so the maximum is taken on the integer
// pipe. Each kernel writes only the fields it owns: the structural update
// runs concurrently and owns flag_pending.
__global__ void k_begin_step(Consts c, Params* prm, const double* __restrict__ partial,
                             int n_partial, double tol, int hmax) {
  __shared__ unsigned long long wmax[32];
  unsigned long long mb = 0ull;
  for (int b = threadIdx.x; b < n_partial; b += blockDim.x)
    mb = max(mb, (unsigned long long)__double_as_longlong(partial[b]));
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mb = max(mb, wmax[q]);
    const double m = __longlong_as_double((long long)mb);
    const double dt_fixed = prm->dt_fixed;
    int err = 0;
    double dt = dt_fixed > 0.0 ? dt_fixed : prm->cfl * c.h / m;
    if (!isfinite(m) || !(dt > 0.0) || !isfinite(dt)) {
      err |= ERR_NONFINITE;
      dt = dt_fixed > 0.0 ? dt_fixed : 1e-300;
    }
    double alpha = 1.0, beta = 0.0;
    if (!prm->first) {
      alpha = 1.0 + dt / (2.0 * prm->dt_old);
      beta = -dt / (2.0 * prm->dt_old);
    }
    double r = c.nu * dt / (2.0 * c.h * c.h);
    if (!(r > 0.0) || !isfinite(r)) {
      err |= ERR_AF_RANGE;
      r = 1e-300;
    }
    const double th = af_theta(r);
    const double rho = exp(-th);
    int H = (int)ceil(log(tol) / log(rho));
    if (!(H >= 1)) H = 1;
    if (H > hmax) {
      err |= ERR_AF_RANGE;
      H = hmax;
    }
    // velocity Verlet is stable for dt_s omega < 2; omega_max is a Gershgorin
    // upper bound, so dt_s = dt / n_sub <= 1.8 / omega_max keeps every mode stable
    const double ns = ceil(dt * c.omega_max / 1.8);
    prm->speed_max = m;
    prm->slip_max = 0.0;
    prm->dt = dt;
    prm->alpha = alpha;
    prm->beta = beta;
    prm->r = r;
    prm->af_rho = rho;
    prm->af_h = H;
    prm->n_sub = ns < 1.0 ? 1 : (ns > 1e6 ? 1000000 : (int)ns);
    prm->f_dt = (float)dt;
    prm->f_alpha = (float)alpha;
    prm->f_beta = (float)beta;
    prm->f_r = (float)r;
    prm->f_ir = (float)(1.0 / r);
    prm->f_rho = (float)rho;
    prm->f_gdt = (float)(dt * c.inv_h);
    prm->f_hnu = (float)(0.5 * c.nu * dt * c.inv_h * c.inv_h);
    prm->f_cc = (float)(c.u_in * dt * c.inv_h);
    prm->f_sc_div = (float)(c.inv_h / dt);
    if (err) prm->error |= err;
  }
}

// After the last step of a call: the speed maximum of the velocity that step
// left (the projection's block partials, reduced as in k_begin_step), so that
// a non-finite or too fast field is reported by the call that produced it
__global__ void k_speed_check(Params* prm, const double* __restrict__ partial, int n_partial) {
  __shared__ unsigned long long wmax[32];
  unsigned long long mb = 0ull;
  for (int b = threadIdx.x; b < n_partial; b += blockDim.x)
    mb = max(mb, (unsigned long long)__double_as_longlong(partial[b]));
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mb = max(mb, wmax[q]);
    const double m = __longlong_as_double((long long)mb);
    prm->speed_max = m;
    if (!isfinite(m)) atomicOr(&prm->error, ERR_NONFINITE);
  }
}

template <class T>
void launch_speed_check(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  (void)c;
  k_speed_check<<<1, 1024, 0, s>>>(f.prm, f.partial, f.n_partial);
}
template void launch_speed_check<float>(const Consts&, const Fields<float>&, cudaStream_t);
template void launch_speed_check<double>(const Consts&, const Fields<double>&, cudaStream_t);

// Tables of the implicit factors for this step's r, one entry per thread
// (FP64 transcendental functions: spread over many blocks, and off the
// critical path, concurrent with the explicit stage):
//   LU inverse pivots of the x factors (closed form)
//     Dirichlet start (u):      1/p_k = rho (1 - rho^{2k})   / (1 - rho^{2k+2})
//     reflection start (v, w):  1/p_k = rho (1 - rho^{2k-1}) / (1 - rho^{2k+1})
//   free-space taps of the reflected x solve: (1/r) rho^{m+1} / (1 - rho^2)
//   taps of the exact periodic inverse of r (q - S - S^{-1}) on n points:
//     t_m = (1/r) rho / (1 - rho^2) (rho^m + rho^{n-m}) / (1 - rho^n)
constexpr int TAB_THREADS = 64;
int table_entries(const Consts& c) { return c.nx + (HMAX + 1) + c.ny + c.nz; }

__global__ void __launch_bounds__(TAB_THREADS)
k_af_tables(Consts c, const Params* __restrict__ prm, double* __restrict__ ipt,
            float* __restrict__ iptf, double* __restrict__ taps, float* __restrict__ tapsf) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  const double r = prm->r;
  const double th = af_theta(r);
  const double rho = exp(-th);
  if (q < c.nx) {
    const int k = q + 1;
    const double a = rho * expm1(-2.0 * k * th) / expm1(-(2.0 * k + 2.0) * th);
    const double b = rho * expm1(-(2.0 * k - 1.0) * th) / expm1(-(2.0 * k + 1.0) * th);
    ipt[k] = a;
    ipt[c.nx + 2 + k] = b;
    iptf[k] = (float)a;
    iptf[c.nx + 2 + k] = (float)b;
    return;
  }
  q -= c.nx;
  if (q <= HMAX) {
    const double v = (1.0 / r) * exp(-(double)(q + 1) * th) / (-expm1(-2.0 * th));
    taps[c.ny + c.nz + q] = v;
    tapsf[c.ny + c.nz + q] = (float)v;
    return;
  }
  q -= HMAX + 1;
  const int dir = q < c.ny ? 0 : 1;
  const int n = dir == 0 ? c.ny : c.nz;
  const int m = dir == 0 ? q : q - c.ny;
  if (m >= n) return;
  const double pre = (1.0 / r) * rho / (-expm1(-2.0 * th));
  const double den = -expm1(-(double)n * th);
  const double v = pre * (exp(-(double)m * th) + exp(-(double)(n - m) * th)) / den;
  taps[q] = v;    // y taps at [0, ny), z taps at [ny, ny + nz)
  tapsf[q] = (float)v;
}

// after the projection: advance the clock
__global__ void k_end_step(Params* prm) {
  prm->t += prm->dt;
  prm->dt_old = prm->dt;
  prm->step += 1;
  prm->first = 0;
}

// ---------------------------------------------------------------- RHS (A2)
// RHS = dt [ -(alpha N^n + beta N^{n-1}) - G p^n + nu L u^n ], N in flux form.
// One thread per (y, z) column and XCHUNK x planes; neighbours through L1.
// column (j, k), x planes i0 .. i1 - 1 (block (bx, by, bz) of the grid
// grid3(c, nx + 1) with threads (TK, TJ))
template <class T>
__device__ inline void rhs_block(const Consts& c, const Params* __restrict__ prm, const T* __restrict__ u,
                                 const T* __restrict__ v, const T* __restrict__ w, const T* __restrict__ p,
                                 T* __restrict__ n0, T* __restrict__ n1, T* __restrict__ n2,
                                 T* __restrict__ d0, T* __restrict__ d1, T* __restrict__ d2,
                                 const T* __restrict__ vin, const T* __restrict__ win, int bx, int by, int bz) {
  const int k = bx * TK + threadIdx.x;
  const int j = by * TJ + threadIdx.y;
  if (k >= c.nz || j >= c.ny) return;
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
  const T dt = pick<T>(prm->dt, prm->f_dt), alpha = pick<T>(prm->alpha, prm->f_alpha);
  const T beta = pick<T>(prm->beta, prm->f_beta);
  const T nu = pick<T>(c.nu, c.f_nu), ih = pick<T>(c.inv_h, c.f_inv_h);
  const T ih2 = pick<T>(c.inv_h * c.inv_h, c.f_inv_h2), hf = (T)0.5;
  const size_t P = plane(c);
  auto at = [&](int i, int jj, int kk) { return ((size_t)i * ny + jj) * nz + kk; };
  const int i0 = bz * XCHUNK;
  const int i1 = min(i0 + XCHUNK, nx + 1);
  for (int i = i0; i < i1; ++i) {
    const size_t id = at(i, j, k);
    if (i >= 1 && i <= nx - 1) {
      const T uc = u[id];
      const T uxp = u[id + P], uxm = u[id - P];
      const T uyp = u[at(i, jp, k)], uym = u[at(i, jm, k)];
      const T uzp = u[at(i, j, kp)], uzm = u[at(i, j, km)];
      T fxp = hf * (uc + uxp);
      fxp *= fxp;
      T fxm = hf * (uxm + uc);
      fxm *= fxm;
      // xy-edges (i, j) and (i, j+1); v is interior on both sides (1 <= i <= nx-1)
      const T fxy0 = hf * (uym + uc) * (hf * (v[at(i - 1, j, k)] + v[id]));
      const T fxy1 = hf * (uc + uyp) * (hf * (v[at(i - 1, jp, k)] + v[at(i, jp, k)]));
      const T fxz0 = hf * (uzm + uc) * (hf * (w[at(i - 1, j, k)] + w[id]));
      const T fxz1 = hf * (uc + uzp) * (hf * (w[at(i - 1, j, kp)] + w[at(i, j, kp)]));
      const T N = (fxp - fxm + fxy1 - fxy0 + fxz1 - fxz0) * ih;
      const T L = (uxp + uxm + uyp + uym + uzp + uzm - (T)6 * uc) * ih2;
      const T Gp = (p[at(i, j, k)] - p[at(i - 1, j, k)]) * ih;
      const T Np = n0[id];
      n0[id] = N;
      d0[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
    }
    if (i <= nx - 1) {
      // ---- v at ((i+1/2) h, j h, (k+1/2) h); inflow ghost v_{-1} = -v_0
      {
        const T vc = v[id];
        const T vxp = v[id + P];
        const T vxm = i == 0 ? (vin ? (T)2 * vin[(size_t)j * nz + k] : (T)0) - vc : v[id - P];
        const T vyp = v[at(i, jp, k)], vym = v[at(i, jm, k)];
        const T vzp = v[at(i, j, kp)], vzm = v[at(i, j, km)];
        const T fxr = hf * (u[at(i + 1, jm, k)] + u[at(i + 1, j, k)]) * (hf * (vc + vxp));
        const T fxl = hf * (u[at(i, jm, k)] + u[id]) * (hf * (vxm + vc));
        T fyp = hf * (vc + vyp);
        fyp *= fyp;
        T fym = hf * (vym + vc);
        fym *= fym;
        const T fz1 = hf * (vc + vzp) * (hf * (w[at(i, jm, kp)] + w[at(i, j, kp)]));
        const T fz0 = hf * (vzm + vc) * (hf * (w[at(i, jm, k)] + w[id]));
        const T N = (fxr - fxl + fyp - fym + fz1 - fz0) * ih;
        const T L = (vxp + vxm + vyp + vym + vzp + vzm - (T)6 * vc) * ih2;
        const T Gp = (p[at(i, j, k)] - p[at(i, jm, k)]) * ih;
        const T Np = n1[id];
        n1[id] = N;
        d1[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
      }
      // ---- w at ((i+1/2) h, (j+1/2) h, k h)
      {
        const T wc = w[id];
        const T wxp = w[id + P];
        const T wxm = i == 0 ? (win ? (T)2 * win[(size_t)j * nz + k] : (T)0) - wc : w[id - P];
        const T wyp = w[at(i, jp, k)], wym = w[at(i, jm, k)];
        const T wzp = w[at(i, j, kp)], wzm = w[at(i, j, km)];
        const T fxr = hf * (u[at(i + 1, j, km)] + u[at(i + 1, j, k)]) * (hf * (wc + wxp));
        const T fxl = hf * (u[at(i, j, km)] + u[id]) * (hf * (wxm + wc));
        const T fy1 = hf * (v[at(i, jp, km)] + v[at(i, jp, k)]) * (hf * (wc + wyp));
        const T fy0 = hf * (v[at(i, j, km)] + v[id]) * (hf * (wym + wc));
        T fzp = hf * (wc + wzp);
        fzp *= fzp;
        T fzm = hf * (wzm + wc);
        fzm *= fzm;
        const T N = (fxr - fxl + fy1 - fy0 + fzp - fzm) * ih;
        const T L = (wxp + wxm + wyp + wym + wzp + wzm - (T)6 * wc) * ih2;
        const T Gp = (p[at(i, j, k)] - p[at(i, j, km)]) * ih;
        const T Np = n2[id];
        n2[id] = N;
        d2[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_rhs(Consts c, const Params* __restrict__ prm, const T* __restrict__ u,
      const T* __restrict__ v, const T* __restrict__ w, const T* __restrict__ p,
      T* __restrict__ n0, T* __restrict__ n1, T* __restrict__ n2, T* __restrict__ d0,
      T* __restrict__ d1, T* __restrict__ d2, const T* __restrict__ vin,
      const T* __restrict__ win) {
  rhs_block<T>(c, prm, u, v, w, p, n0, n1, n2, d0, d1, d2, vin, win, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The explicit stage of several independent cases (an ensemble) in one
// persistent launch: the case table lists per case its constants, fields
// and block grid; the blocks of the launch walk the concatenated block
// lists of all cases.
template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_rhs_cases(const RhsCase<T>* __restrict__ table, int ncases, int total) {
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int q = 0;
    while (q + 1 < ncases && table[q + 1].first <= item) ++q;
    const RhsCase<T>& e = table[q];
    const int local = item - e.first;
    const int bx = local % e.gx, by = (local / e.gx) % e.gy, bz = local / (e.gx * e.gy);
    rhs_block<T>(e.c, e.prm, e.u, e.v, e.w, e.p, e.n0, e.n1, e.n2, e.d0, e.d1, e.d2, e.vin, e.win, bx, by, bz);
  }
}

// Pipelined RHS (same arithmetic as k_rhs): a block owns TJ whole z-rows
// of y and marches XR x-planes. For every x plane one thread issues bulk
// asynchronous copies (TMA engine) of the rows j0-1 .. j0+TJ of u, v, w and
// j0-1 .. j0+TJ-1 of p into a STAGES-deep shared-memory ring, completing on
// one mbarrier per slot; the block computes plane i from planes i-1, i, i+1
// while the copies of the next planes are in flight. Whole rows make the
// periodic z wrap an index mask and every copy 16-byte aligned.
constexpr int RSTAGES_MAX = 8;   // ring slots: as many stages as 210 KB holds, 4..8
template <class T, int TJR>
struct RhsRing {
  // rows of one stage: u, v, w with halo, p with low-side halo, N^{n-1} x 3
  static constexpr int ROWS = 3 * (TJR + 2) + (TJR + 1) + 3 * TJR;
};
constexpr int RTHREADS = 512;

template <class T, int TJR>
__global__ void __launch_bounds__(RTHREADS, 1)
k_rhs_pipe(Consts c, Params* __restrict__ prm, const T* __restrict__ u,
           const T* __restrict__ v, const T* __restrict__ w, const T* __restrict__ p,
           T* __restrict__ n0, T* __restrict__ n1, T* __restrict__ n2, T* __restrict__ d0,
           T* __restrict__ d1, T* __restrict__ d2, int XR, int RSTAGES, const T* __restrict__ vin,
           const T* __restrict__ win) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t full[RSTAGES_MAX];
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * TJR;
  const int ib = blockIdx.y * XR, ie = min(ib + XR, nx);
  const size_t P = plane(c);
  const size_t rowb = (size_t)nz * sizeof(T);
  constexpr int RW = TJR + 2;          // rows of u, v, w in a stage
  constexpr int ROWS = RhsRing<T, TJR>::ROWS;
  T* ring = reinterpret_cast<T*>(smem_raw);
  auto stage_ptr = [&](int slot) { return ring + (size_t)slot * ROWS * nz; };
  // stage t holds x plane q = ib - 1 + t (t = 0 .. ie - ib + 1)
  const int nstage = ie - ib + 2;
  auto issue = [&](int t) {
    const int q = ib - 1 + t;
    const int qs = q < 0 ? 0 : q;
    const bool has_p = (q >= 0 && q <= nx - 1);
    const int slot = t % RSTAGES;
    T* st = stage_ptr(slot);
    const uint32_t bytes = (uint32_t)((3 * RW + (has_p ? (TJR + 1) + 3 * TJR : 0)) * rowb);
    mbar_arrive_expect_tx(&full[slot], bytes);
    for (int r = 0; r < RW; ++r) {
      int jj = j0 - 1 + r;
      jj = jj < 0 ? jj + ny : (jj >= ny ? jj - ny : jj);
      const size_t g = ((size_t)qs * ny + jj) * nz;
      bulk_g2s(st + (size_t)r * nz, u + g, (uint32_t)rowb, &full[slot]);
      bulk_g2s(st + (size_t)(RW + r) * nz, v + g, (uint32_t)rowb, &full[slot]);
      bulk_g2s(st + (size_t)(2 * RW + r) * nz, w + g, (uint32_t)rowb, &full[slot]);
    }
    if (has_p) {
      for (int r = 0; r < TJR + 1; ++r) {
        int jj = j0 - 1 + r;
        jj = jj < 0 ? jj + ny : jj;
        bulk_g2s(st + (size_t)(3 * RW + r) * nz, p + ((size_t)q * ny + jj) * nz, (uint32_t)rowb,
                 &full[slot]);
      }
      const int nb = 3 * RW + TJR + 1;
      for (int r = 0; r < TJR; ++r) {
        const size_t g = ((size_t)q * ny + j0 + r) * nz;
        bulk_g2s(st + (size_t)(nb + r) * nz, n0 + g, (uint32_t)rowb, &full[slot]);
        bulk_g2s(st + (size_t)(nb + TJR + r) * nz, n1 + g, (uint32_t)rowb, &full[slot]);
        bulk_g2s(st + (size_t)(nb + 2 * TJR + r) * nz, n2 + g, (uint32_t)rowb, &full[slot]);
      }
    }
  };
  if (tid == 0) {
    for (int sl = 0; sl < RSTAGES; ++sl) mbar_init(&full[sl], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < RSTAGES && t < nstage; ++t) issue(t);
  const T dt = pick<T>(prm->dt, prm->f_dt), alpha = pick<T>(prm->alpha, prm->f_alpha);
  const T beta = pick<T>(prm->beta, prm->f_beta);
  const T nu = pick<T>(c.nu, c.f_nu), ih = pick<T>(c.inv_h, c.f_inv_h);
  const T ih2 = pick<T>(c.inv_h * c.inv_h, c.f_inv_h2), hf = (T)0.5;
  const int mask = nz - 1;
  const int ncell = TJR * nz;
  const int lg = __ffs(nz) - 1;
  // stage t is ready when its slot's barrier completed use number t / RSTAGES
  auto wait_stage = [&](int t) {
    return mbar_wait(&full[t % RSTAGES], (uint32_t)((t / RSTAGES) & 1));
  };
  bool ok = wait_stage(0) && wait_stage(1);
  for (int i = ib; i < ie; ++i) {
    const int ta = i - ib, tb = ta + 1, tc = ta + 2;
    ok = ok && wait_stage(tc);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&prm->error, ERR_TIMEOUT);
        // let the copies already issued land before the block leaves
        // (issued so far: stages up to ta - 1 + RSTAGES)
        for (int t = tc; t < nstage && t < ta + RSTAGES; ++t) (void)wait_stage(t);
      }
      return;
    }
    const T* A = stage_ptr(ta % RSTAGES);
    const T* B = stage_ptr(tb % RSTAGES);
    const T* C = stage_ptr(tc % RSTAGES);
    const T sgn = i - 1 < 0 ? (T)-1 : (T)1;   // inflow reflection ghost of v, w
    for (int cidx = tid; cidx < ncell; cidx += blockDim.x) {
      const int r = cidx >> lg, k = cidx & mask;
      const int j = j0 + r;
      if (j >= ny) continue;
      const int kp = (k + 1) & mask, km = (k - 1) & mask;
      const int R = (r + 1) * nz, Rm = r * nz, Rp = (r + 2) * nz;
      // row pointers: U, V, W planes a (i-1), b (i), c (i+1); P planes a, b
      const T* Ua = A;
      const T* Ub = B;
      const T* Uc = C;
      const T* Va = A + RW * nz;
      const T* Vb = B + RW * nz;
      const T* Vc = C + RW * nz;
      const T* Wa = A + 2 * RW * nz;
      const T* Wb = B + 2 * RW * nz;
      const T* Wc = C + 2 * RW * nz;
      const T* Pa = A + 3 * RW * nz;
      const T* Pb = B + 3 * RW * nz;
      const T* Nb = B + (3 * RW + TJR + 1) * nz + r * nz + k;   // N^{n-1} of plane i
      const size_t id = ((size_t)i * ny + j) * nz + k;
      const T pc = Pb[R + k];
      if (i >= 1) {
        const T uc = Ub[R + k];
        const T uxp = Uc[R + k], uxm = Ua[R + k];
        const T uyp = Ub[Rp + k], uym = Ub[Rm + k];
        const T uzp = Ub[R + kp], uzm = Ub[R + km];
        T fxp = hf * (uc + uxp);
        fxp *= fxp;
        T fxm = hf * (uxm + uc);
        fxm *= fxm;
        const T fxy0 = hf * (uym + uc) * (hf * (sgn * Va[R + k] + Vb[R + k]));
        const T fxy1 = hf * (uc + uyp) * (hf * (sgn * Va[Rp + k] + Vb[Rp + k]));
        const T fxz0 = hf * (uzm + uc) * (hf * (sgn * Wa[R + k] + Wb[R + k]));
        const T fxz1 = hf * (uc + uzp) * (hf * (sgn * Wa[R + kp] + Wb[R + kp]));
        const T N = (fxp - fxm + fxy1 - fxy0 + fxz1 - fxz0) * ih;
        const T L = (uxp + uxm + uyp + uym + uzp + uzm - (T)6 * uc) * ih2;
        const T Gp = (pc - Pa[R + k]) * ih;
        const T Np = Nb[0];
        n0[id] = N;
        d0[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
      }
      {
        const T vc = Vb[R + k];
        const T vxp = Vc[R + k];
        const T vxm = sgn * Va[R + k] + ((i == 0 && vin) ? (T)2 * vin[(size_t)j * nz + k] : (T)0);
        const T vyp = Vb[Rp + k], vym = Vb[Rm + k];
        const T vzp = Vb[R + kp], vzm = Vb[R + km];
        const T fxr = hf * (Uc[Rm + k] + Uc[R + k]) * (hf * (vc + vxp));
        const T fxl = hf * (Ub[Rm + k] + Ub[R + k]) * (hf * (vxm + vc));
        T fyp = hf * (vc + vyp);
        fyp *= fyp;
        T fym = hf * (vym + vc);
        fym *= fym;
        const T fz1 = hf * (vc + vzp) * (hf * (Wb[Rm + kp] + Wb[R + kp]));
        const T fz0 = hf * (vzm + vc) * (hf * (Wb[Rm + k] + Wb[R + k]));
        const T N = (fxr - fxl + fyp - fym + fz1 - fz0) * ih;
        const T L = (vxp + vxm + vyp + vym + vzp + vzm - (T)6 * vc) * ih2;
        const T Gp = (pc - Pb[Rm + k]) * ih;
        const T Np = Nb[TJR * nz];
        n1[id] = N;
        d1[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
      }
      {
        const T wc = Wb[R + k];
        const T wxp = Wc[R + k];
        const T wxm = sgn * Wa[R + k] + ((i == 0 && win) ? (T)2 * win[(size_t)j * nz + k] : (T)0);
        const T wyp = Wb[Rp + k], wym = Wb[Rm + k];
        const T wzp = Wb[R + kp], wzm = Wb[R + km];
        const T fxr = hf * (Uc[R + km] + Uc[R + k]) * (hf * (wc + wxp));
        const T fxl = hf * (Ub[R + km] + Ub[R + k]) * (hf * (wxm + wc));
        const T fy1 = hf * (Vb[Rp + km] + Vb[Rp + k]) * (hf * (wc + wyp));
        const T fy0 = hf * (Vb[R + km] + Vb[R + k]) * (hf * (wym + wc));
        T fzp = hf * (wc + wzp);
        fzp *= fzp;
        T fzm = hf * (wzm + wc);
        fzm *= fzm;
        const T N = (fxr - fxl + fy1 - fy0 + fzp - fzm) * ih;
        const T L = (wxp + wxm + wyp + wym + wzp + wzm - (T)6 * wc) * ih2;
        const T Gp = (pc - Pb[R + km]) * ih;
        const T Np = Nb[2 * TJR * nz];
        n2[id] = N;
        d2[id] = dt * (-(alpha * N + beta * Np) - Gp + nu * L);
      }
    }
    __syncthreads();
    // the slot of plane i-1 is free: refill it with the stage RSTAGES ahead
    if (tid == 0 && ta + RSTAGES < nstage) issue(ta + RSTAGES);
  }
}

// Streamed explicit stage, vector form. Same arithmetic as above; each thread
// owns a run of E = 16 / sizeof(T) consecutive z points of one row and reads
// its stencil rows with 16-byte shared loads (plus single values at the run's
// two z edges), so a cell costs about eight shared loads instead of ~34.
// The ring stages u, v, w (rows j0-1 .. j0+TJ) and p (rows j0-1 .. j0+TJ-1)
// of one x plane per slot; N^{n-1} is read straight from global memory into
// registers (it has no neighbours in the stencil). A block is TJ rows of
// runs (256 threads at nz = 256); FP32 fits two blocks per SM.
template <class T>
struct RhsVec {
  static constexpr int E = 16 / sizeof(T);
  static constexpr int TJ = sizeof(T) == 4 ? 4 : 2;
  static constexpr int RW = TJ + 2;
  static constexpr int ROWS = 3 * RW + TJ + 1;
  static constexpr int STAGES = 4;
};
template <class T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
};
template <>
struct V16<double> {
  using type = double2;
};
template <class T, int E>
__device__ inline void lds_run(const T* p, T (&v)[E]) {
  const typename V16<T>::type q = *reinterpret_cast<const typename V16<T>::type*>(p);
  if constexpr (E == 4) {
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    v[0] = q.x;
    v[1] = q.y;
  }
}
template <class T, int E>
__device__ inline void stg_run(T* p, const T (&v)[E]) {
  using V = typename V16<T>::type;
  if constexpr (E == 4) {
    *reinterpret_cast<V*>(p) = V{v[0], v[1], v[2], v[3]};
  } else {
    *reinterpret_cast<V*>(p) = V{v[0], v[1]};
  }
}
template <class T, int E>
__device__ inline void ldg_run(const T* p, T (&v)[E]) {
  lds_run<T, E>(p, v);
}

template <class T>
__global__ void __launch_bounds__(256, 2)
k_rhs_vec(Consts c, Params* __restrict__ prm, const T* __restrict__ u, const T* __restrict__ v,
          const T* __restrict__ w, const T* __restrict__ p, T* __restrict__ n0,
          T* __restrict__ n1, T* __restrict__ n2, T* __restrict__ d0, T* __restrict__ d1,
          T* __restrict__ d2, int XR, const T* __restrict__ vin, const T* __restrict__ win) {
  using RV = RhsVec<T>;
  constexpr int E = RV::E, TJ = RV::TJ, RW = RV::RW, ROWS = RV::ROWS, NS = RV::STAGES;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t full[NS];
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * TJ;
  const int ib = blockIdx.y * XR, ie = min(ib + XR, nx);
  const size_t rowb = (size_t)nz * sizeof(T);
  T* ring = reinterpret_cast<T*>(smem_raw);
  auto stage_ptr = [&](int slot) { return ring + (size_t)slot * ROWS * nz; };
  const int nstage = ie - ib + 2;   // stage t holds x plane ib - 1 + t
  auto issue = [&](int t) {
    const int q = ib - 1 + t;
    const int qs = q < 0 ? 0 : q;
    const bool has_p = (q >= 0 && q <= nx - 1);
    const int slot = t % NS;
    T* st = stage_ptr(slot);
    const uint32_t bytes = (uint32_t)((3 * RW + (has_p ? TJ + 1 : 0)) * rowb);
    mbar_arrive_expect_tx(&full[slot], bytes);
    for (int r = 0; r < RW; ++r) {
      int jj = j0 - 1 + r;
      jj = jj < 0 ? jj + ny : (jj >= ny ? jj - ny : jj);
      const size_t g = ((size_t)qs * ny + jj) * nz;
      bulk_g2s(st + (size_t)r * nz, u + g, (uint32_t)rowb, &full[slot]);
      bulk_g2s(st + (size_t)(RW + r) * nz, v + g, (uint32_t)rowb, &full[slot]);
      bulk_g2s(st + (size_t)(2 * RW + r) * nz, w + g, (uint32_t)rowb, &full[slot]);
    }
    if (has_p)
      for (int r = 0; r < TJ + 1; ++r) {
        int jj = j0 - 1 + r;
        jj = jj < 0 ? jj + ny : jj;
        bulk_g2s(st + (size_t)(3 * RW + r) * nz, p + ((size_t)q * ny + jj) * nz, (uint32_t)rowb,
                 &full[slot]);
      }
  };
  const int lane = tid & 31;
  if (tid == 0) {
    for (int sl = 0; sl < NS; ++sl) mbar_init(&full[sl], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < NS && t < nstage; ++t) issue(t);
  const T dt = pick<T>(prm->dt, prm->f_dt), alpha = pick<T>(prm->alpha, prm->f_alpha);
  const T beta = pick<T>(prm->beta, prm->f_beta);
  const T nu = pick<T>(c.nu, c.f_nu), ih = pick<T>(c.inv_h, c.f_inv_h);
  const T ih2 = pick<T>(c.inv_h * c.inv_h, c.f_inv_h2);
  const T qh = (T)0.25 * ih, cdn = dt * nu * ih2, cdg = dt * ih;
  const T mda = -dt * alpha, mdb = -dt * beta;
  const int mask = nz - 1;
  const int runs = nz / E;                  // runs per row
  const int r = tid / runs;                 // row of this thread in the tile
  const int k0 = (tid - r * runs) * E;      // first z point of the run
  const int km1 = (k0 - 1) & mask, kpE = (k0 + E) & mask;
  const int j = j0 + r;
  const int R = (r + 1) * nz, Rm = r * nz, Rp = (r + 2) * nz;   // rows in u, v, w, p blocks
  auto wait_stage = [&](int t) {
    return mbar_wait(&full[t % NS], (uint32_t)((t / NS) & 1));
  };
  bool ok = wait_stage(0) && wait_stage(1);
  // z neighbours across the runs of one row: from the adjacent lane, or read
  // from shared memory at the row's ends and at warp edges
  auto left = [&](T last, const T* row) {
    T v = __shfl_up_sync(0xffffffffu, last, 1);
    if (lane == 0 || k0 == 0) v = row[km1];
    return v;
  };
  auto right = [&](T first, const T* row) {
    T v = __shfl_down_sync(0xffffffffu, first, 1);
    if (lane == 31 || k0 + E >= nz) v = row[kpE];
    return v;
  };
  for (int i = ib; i < ie; ++i) {
    const int ta = i - ib, tb = ta + 1, tc = ta + 2;
    const size_t id = ((size_t)i * ny + j) * nz + k0;
    T Np0[E], Np1[E], Np2[E];
    ldg_run<T, E>(n0 + id, Np0);
    ldg_run<T, E>(n1 + id, Np1);
    ldg_run<T, E>(n2 + id, Np2);
    ok = ok && wait_stage(tc);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&prm->error, ERR_TIMEOUT);
        // let the copies already issued (stages up to ta - 1 + NS) land first
        for (int t = tc; t < nstage && t < ta + NS; ++t) (void)wait_stage(t);
      }
      return;
    }
    const T* A = stage_ptr(ta % NS);
    const T* B = stage_ptr(tb % NS);
    const T* C = stage_ptr(tc % NS);
    const T* Ua = A;
    const T* Ub = B;
    const T* Uc = C;
    const T* Va = A + RW * nz;
    const T* Vb = B + RW * nz;
    const T* Vc = C + RW * nz;
    const T* Wa = A + 2 * RW * nz;
    const T* Wb = B + 2 * RW * nz;
    const T* Wc = C + 2 * RW * nz;
    const T* Pa = A + 3 * RW * nz;
    const T* Pb = B + 3 * RW * nz;
    const T sgn = i - 1 < 0 ? (T)-1 : (T)1;   // inflow ghost of v, w: 2 q_in - q_0
    T gv[E], gw[E];
#pragma unroll
    for (int e = 0; e < E; ++e) gv[e] = gw[e] = (T)0;
    if (i == 0 && vin) {
      ldg_run<T, E>(vin + (size_t)j * nz + k0, gv);
      ldg_run<T, E>(win + (size_t)j * nz + k0, gw);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        gv[e] *= (T)2;
        gw[e] *= (T)2;
      }
    }
    // shared rows of the run (E values) and edge values
    T ub[E], ubm[E], ubp[E], uc[E], ucm[E];
    T vb[E], vbm[E], vbp[E], va[E], vap[E], vc[E];
    T wb[E], wbm[E], wbp[E], wa[E], wc[E];
    T pb[E], pbm[E];
    lds_run<T, E>(Ub + R + k0, ub);
    lds_run<T, E>(Ub + Rm + k0, ubm);
    lds_run<T, E>(Ub + Rp + k0, ubp);
    lds_run<T, E>(Uc + R + k0, uc);
    lds_run<T, E>(Uc + Rm + k0, ucm);
    lds_run<T, E>(Vb + R + k0, vb);
    lds_run<T, E>(Vb + Rm + k0, vbm);
    lds_run<T, E>(Vb + Rp + k0, vbp);
    lds_run<T, E>(Va + R + k0, va);
    lds_run<T, E>(Va + Rp + k0, vap);
    lds_run<T, E>(Vc + R + k0, vc);
    lds_run<T, E>(Wb + R + k0, wb);
    lds_run<T, E>(Wb + Rm + k0, wbm);
    lds_run<T, E>(Wb + Rp + k0, wbp);
    lds_run<T, E>(Wa + R + k0, wa);
    lds_run<T, E>(Wc + R + k0, wc);
    lds_run<T, E>(Pb + R + k0, pb);
    lds_run<T, E>(Pb + Rm + k0, pbm);
    const T ub_l = left(ub[E - 1], Ub + R), ub_r = right(ub[0], Ub + R);
    const T uc_l = left(uc[E - 1], Uc + R);
    const T vb_l = left(vb[E - 1], Vb + R), vb_r = right(vb[0], Vb + R);
    const T vbp_l = left(vbp[E - 1], Vb + Rp);
    const T wb_l = left(wb[E - 1], Wb + R), wb_r = right(wb[0], Wb + R);
    const T wa_r = right(wa[0], Wa + R), wbm_r = right(wbm[0], Wb + Rm);
    const T pb_l = left(pb[E - 1], Pb + R);
    T No[E], Do[E];
    // Flux differences with the halves folded into qh = ih / 4:
    // (a+b)/2 (c+d)/2 products become (a+b)(c+d), and each face pair is one
    // product and one fused multiply-add. RHS = -dt alpha N - dt beta N^{n-1}
    // + dt nu ih^2 Lraw - dt ih (p_c - p_w), every term one FMA.
    // u on face i (interior faces only; no inflow ghost enters it)
    if (i >= 1) {
      T ua[E], pa[E];
      lds_run<T, E>(Ua + R + k0, ua);
      lds_run<T, E>(Pa + R + k0, pa);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const T c0 = ub[e];
        const T uzp = e == E - 1 ? ub_r : ub[e + 1], uzm = e == 0 ? ub_l : ub[e - 1];
        const T wap = e == E - 1 ? wa_r : wa[e + 1], wbp1 = e == E - 1 ? wb_r : wb[e + 1];
        const T sp = c0 + uc[e], sm = ua[e] + c0;
        const T fx = sp * sp - sm * sm;
        const T fy = (c0 + ubp[e]) * (vap[e] + vbp[e]) - (ubm[e] + c0) * (va[e] + vb[e]);
        const T fz = (c0 + uzp) * (wap + wbp1) - (uzm + c0) * (wa[e] + wb[e]);
        const T N = qh * (fx + fy + fz);
        const T L = uc[e] + ua[e] + ubp[e] + ubm[e] + uzp + uzm - (T)6 * c0;
        No[e] = N;
        Do[e] = mda * N + (mdb * Np0[e] + (cdn * L - cdg * (pb[e] - pa[e])));
      }
      stg_run<T, E>(n0 + id, No);
      stg_run<T, E>(d0 + id, Do);
    }
    // v at (i + 1/2, j, k + 1/2)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T c0 = vb[e];
      const T vxp = vc[e], vxm = sgn * va[e] + gv[e];
      const T vzp = e == E - 1 ? vb_r : vb[e + 1], vzm = e == 0 ? vb_l : vb[e - 1];
      const T wbp1 = e == E - 1 ? wb_r : wb[e + 1], wbmp1 = e == E - 1 ? wbm_r : wbm[e + 1];
      const T fx = (ucm[e] + uc[e]) * (c0 + vxp) - (ubm[e] + ub[e]) * (vxm + c0);
      const T sp = c0 + vbp[e], sm = vbm[e] + c0;
      const T fy = sp * sp - sm * sm;
      const T fz = (c0 + vzp) * (wbmp1 + wbp1) - (vzm + c0) * (wbm[e] + wb[e]);
      const T N = qh * (fx + fy + fz);
      const T L = vxp + vxm + vbp[e] + vbm[e] + vzp + vzm - (T)6 * c0;
      No[e] = N;
      Do[e] = mda * N + (mdb * Np1[e] + (cdn * L - cdg * (pb[e] - pbm[e])));
    }
    stg_run<T, E>(n1 + id, No);
    stg_run<T, E>(d1 + id, Do);
    // w at (i + 1/2, j + 1/2, k)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T c0 = wb[e];
      const T wxp = wc[e], wxm = sgn * wa[e] + gw[e];
      const T wzp = e == E - 1 ? wb_r : wb[e + 1], wzm = e == 0 ? wb_l : wb[e - 1];
      const T ucl = e == 0 ? uc_l : uc[e - 1], ubl = e == 0 ? ub_l : ub[e - 1];
      const T vbpl = e == 0 ? vbp_l : vbp[e - 1], vbl = e == 0 ? vb_l : vb[e - 1];
      const T pbl = e == 0 ? pb_l : pb[e - 1];
      const T fx = (ucl + uc[e]) * (c0 + wxp) - (ubl + ub[e]) * (wxm + c0);
      const T fy = (vbpl + vbp[e]) * (c0 + wbp[e]) - (vbl + vb[e]) * (wbm[e] + c0);
      const T sp = c0 + wzp, sm = wzm + c0;
      const T fz = sp * sp - sm * sm;
      const T N = qh * (fx + fy + fz);
      const T L = wxp + wxm + wbp[e] + wbm[e] + wzp + wzm - (T)6 * c0;
      No[e] = N;
      Do[e] = mda * N + (mdb * Np2[e] + (cdn * L - cdg * (pb[e] - pbl)));
    }
    stg_run<T, E>(n2 + id, No);
    stg_run<T, E>(d2 + id, Do);
    __syncthreads();
    // the slot of plane i-1 is free: refill it with the stage NS ahead
    if (tid == 0 && ta + NS < nstage) issue(ta + NS);
  }
}

// ---------------------------------------------------------------- outflow (A1)
// Convective condition dq/dt + U dq/dx = 0 on the outflow plane, first-order
// upwind; the increment is kept for the x line solve. The inflow and new
// outflow face fluxes are summed per block in FP64 (fixed order) for the
// mass fix; the IB forcing never touches these two planes.
constexpr int OUT_THREADS = 256;
template <class T>
__global__ void __launch_bounds__(OUT_THREADS)
k_outflow(Consts c, const Params* __restrict__ prm, T* __restrict__ u,
          T* __restrict__ v, T* __restrict__ w, T* __restrict__ o0, T* __restrict__ o1,
          T* __restrict__ o2, double* __restrict__ qpart) {
  __shared__ double scratch[32];
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = c.ny * c.nz;
  double qi = 0.0, qo = 0.0;
  if (jk < P) {
    const T cc = pick<T>(c.u_in * prm->dt * c.inv_h, prm->f_cc);
    const size_t last = (size_t)c.nx * P + jk, prev = last - P;
    T inc = -cc * (u[last] - u[prev]);
    const T un = u[last] + inc;
    u[last] = un;
    o0[jk] = inc;
    inc = -cc * (v[last] - v[prev]);
    v[last] += inc;
    o1[jk] = inc;
    inc = -cc * (w[last] - w[prev]);
    w[last] += inc;
    o2[jk] = inc;
    qi = (double)u[jk];
    qo = (double)un;
  }
  qi = block_sum(qi, scratch);
  __syncthreads();
  qo = block_sum(qo, scratch);
  if (threadIdx.x == 0) {
    qpart[2 * blockIdx.x] = qi;
    qpart[2 * blockIdx.x + 1] = qo;
  }
}

// asynchronous copy of one element (4 or 8 bytes) into shared memory
template <class T>
__device__ inline void cp_async_elem(uint32_t dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(sizeof(T)) : "memory");
}

// x factor by the LU recursions on shared-memory-staged planes: one warp per
// 32 consecutive (y, z) columns and XS planes (+ warm-up halos); lanes walk
// their columns (bank-conflict free), loads and stores are 128-byte rows.
template <class T, int XS>
__global__ void __launch_bounds__(32)
k_af_xr(Consts c, const Params* __restrict__ prm, const T* __restrict__ ipt,
        const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
        T* __restrict__ e0, T* __restrict__ e1, T* __restrict__ e2, const T* __restrict__ o0,
        const T* __restrict__ o1, const T* __restrict__ o2, const T* __restrict__ inc) {
  __shared__ T s[(XS + 2 * hmax_of<T>()) * 32];
  const int P = c.ny * c.nz;
  const int lane = threadIdx.x;
  const int col0 = blockIdx.x * 32;
  const int comp = blockIdx.z;
  const int m = comp == 0 ? c.nx - 1 : c.nx;   // unknowns k = 1..m
  const int ioff = comp == 0 ? 0 : -1;         // plane i = k + ioff
  const int k0 = 1 + blockIdx.y * XS;
  if (k0 > m) return;
  const int k1 = min(k0 + XS, m + 1);
  const int H = prm->af_h;
  const int ks = max(1, k0 - H), ke = min(m, k1 - 1 + H);
  const T* ip = ipt + (comp == 0 ? 0 : c.nx + 2);
  const T ir = pick<T>(1.0 / prm->r, prm->f_ir);
  const int col = col0 + lane;
  const bool act = col < P;
  const T* d = (comp == 0 ? d0 : comp == 1 ? d1 : d2) + (size_t)ioff * P + col;
  T* out = (comp == 0 ? e0 : comp == 1 ? e1 : e2) + (size_t)ioff * P + col;
  const T ob = act ? (comp == 0 ? o0 : comp == 1 ? o1 : o2)[col] : (T)0;
  // inflow-face increment (u) or twice the inflow-value increment (v, w ghost)
  const T ib = (act && inc) ? (comp == 0 ? (T)1 : (T)2) * inc[(size_t)comp * P + col] : (T)0;
  // every lane copies its column of every plane with cp.async (each warp
  // instruction one coalesced 128-byte row through the load/store path), all
  // planes in flight at once; per-row bulk copies of 128 bytes were limited by
  // the copy engine's issue rate
  if (act) {
    const uint32_t sb = smem_u32(s) + (uint32_t)(lane * sizeof(T));
#pragma unroll 4
    for (int k = ks; k <= ke; ++k)
      cp_async_elem<T>(sb + (uint32_t)((k - ks) * 32 * sizeof(T)), d + (size_t)k * P);
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncwarp();
  if (!act) return;
  // The recursions' loads (plane values, pivots) do not depend on the
  // running value: unrolled, they issue ahead of the two-operation chain.
  // The boundary rows 1 and m are peeled off, so the loops carry no tests.
  // Past the first rows the LU pivots have converged to rho to the last bit
  // (they differ from it by rho^(2k) relative): a segment whose warm-up
  // starts beyond row 32 takes one register for all of them.
  T* sl = s + lane;   // row k at sl[(k - ks) * 32]
  const bool pconst = ks > 32;
  const T ipc = ip[ks];
  auto piv = [&](int k) { return pconst ? ipc : ip[k]; };
  T y = 0;
  int kf = ks;
  if (ks == 1) {
    y = (sl[0] * ir + ib) * ip[1];
    sl[0] = y;
    kf = 2;
  }
  const int kl = ke == m ? m - 1 : ke;   // the last row of the plain loop
#pragma unroll 8
  for (int k = kf; k <= kl; ++k) {
    y = (sl[(k - ks) * 32] * ir + y) * piv(k);
    sl[(k - ks) * 32] = y;
  }
  if (ke == m) {
    y = (sl[(m - ks) * 32] * ir + ob + y) * piv(m);
    sl[(m - ks) * 32] = y;
  }
  T x = 0;
#pragma unroll 8
  for (int k = ke; k >= k1; --k) x = sl[(k - ks) * 32] + x * piv(k);   // warm-up rows
  T* o = out + (size_t)(k1 - 1) * P;
#pragma unroll 8
  for (int k = k1 - 1; k >= k0; --k) {
    x = sl[(k - ks) * 32] + x * piv(k);
    *o = x;
    o -= P;
  }
}

// x factor in registers: one thread per (y, z) column and XV planes, warm-up
// halos of H planes on both sides (the LU recursions forget their start
// within rho^H). Inputs of the segment and of the trailing halo are held in
// registers for the backward pass; 256 columns per block, every access a
// coalesced row of the block's columns.
template <class T, int XV>
__global__ void __launch_bounds__(256)
k_af_xv(Consts c, const Params* __restrict__ prm, const T* __restrict__ ipt,
        const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
        T* __restrict__ e0, T* __restrict__ e1, T* __restrict__ e2, const T* __restrict__ o0,
        const T* __restrict__ o1, const T* __restrict__ o2, const T* __restrict__ inc) {
  const int P = c.ny * c.nz;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const int comp = blockIdx.z;
  const int m = comp == 0 ? c.nx - 1 : c.nx;   // unknowns k = 1..m
  const int ioff = comp == 0 ? 0 : -1;         // plane i = k + ioff
  const int k0 = 1 + blockIdx.y * XV;
  if (k0 > m || col >= P) return;
  const int k1 = min(k0 + XV, m + 1);
  const int H = prm->af_h;
  const int ks = max(1, k0 - H), ke = min(m, k1 - 1 + H);
  const T* ip = ipt + (comp == 0 ? 0 : c.nx + 2);
  const T ir = pick<T>(1.0 / prm->r, prm->f_ir);
  const T* d = (comp == 0 ? d0 : comp == 1 ? d1 : d2) + (size_t)ioff * P + col;
  T* out = (comp == 0 ? e0 : comp == 1 ? e1 : e2) + (size_t)ioff * P + col;
  const T ob = (comp == 0 ? o0 : comp == 1 ? o1 : o2)[col];
  const T ib = inc ? (comp == 0 ? (T)1 : (T)2) * inc[(size_t)comp * P + col] : (T)0;
  // forward warm-up over ks .. k0-1 (values not kept)
  T y = 0;
  for (int kb = ks; kb < k0; kb += 8) {
    T buf[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) buf[t] = (kb + t < k0) ? d[(size_t)(kb + t) * P] : (T)0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (kb + t < k0) y = (buf[t] * ir + (kb + t == 1 ? ib : (T)0) + y) * ip[kb + t];
  }
  // the segment
  const int ns = k1 - k0;
  T yr[XV];
#pragma unroll
  for (int q = 0; q < XV; ++q) yr[q] = q < ns ? d[(size_t)(k0 + q) * P] : (T)0;
#pragma unroll
  for (int q = 0; q < XV; ++q)
    if (q < ns) {
      const int k = k0 + q;
      T e = yr[q] * ir;
      if (k == m) e += ob;
      if (k == 1) e += ib;
      y = (e + y) * ip[k];
      yr[q] = y;
    }
  // trailing halo k1 .. ke, kept for the backward pass
  const int nt = ke - k1 + 1;
  T yt[HMAX];
#pragma unroll
  for (int m0 = 0; m0 < HMAX; m0 += 8) {
    if (m0 < nt) {
      T buf[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[t] = (m0 + t < nt) ? d[(size_t)(k1 + m0 + t) * P] : (T)0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int k = k1 + m0 + t;
        if (m0 + t < nt) {
          T e = buf[t] * ir;
          if (k == m) e += ob;
          if (k == 1) e += ib;
          y = (e + y) * ip[k];
        }
        yt[m0 + t] = y;
      }
    }
  }
  T x = 0;
#pragma unroll
  for (int m0 = HMAX - 8; m0 >= 0; m0 -= 8) {
    if (m0 < nt) {
#pragma unroll
      for (int t = 7; t >= 0; --t)
        if (m0 + t < nt) x = yt[m0 + t] + x * ip[k1 + m0 + t];
    }
  }
#pragma unroll
  for (int q = XV - 1; q >= 0; --q)
    if (q < ns) {
      const int k = k0 + q;
      x = yr[q] + x * ip[k];
      out[(size_t)k * P] = x;
    }
}

// periodic segment solve; in(j), store(j, x) address the line
template <class T, class In, class Out>
__device__ inline void periodic_segment(int n, int j0, int j1, int H, T rho, T ir, In in, Out store) {
  T y = 0;
  int j = (j0 - H) % n;
  if (j < 0) j += n;
  for (int q = 0; q < H; ++q) {
    y = in(j) * ir + rho * y;
    if (++j == n) j = 0;
  }
  // j == j0 here
  const int len = j1 - j0 + H;   // stored forward values
  T yr[SEG + HMAX];
#pragma unroll
  for (int q = 0; q < SEG + HMAX; ++q) {
    if (q < len) {
      y = in(j) * ir + rho * y;
      yr[q] = y;
      if (++j == n) j = 0;
    }
  }
  T z = 0;
#pragma unroll
  for (int q = SEG + HMAX - 1; q >= 0; --q) {
    if (q < len) {
      z = yr[q] + rho * z;
      if (q < j1 - j0) store(j0 + q, rho * z);
    }
  }
}

// y lines: threads over (k, segment), walking y with stride nz (coalesced in k)
template <class T>
__global__ void __launch_bounds__(128)
k_af_y(Consts c, const Params* __restrict__ prm, const T* __restrict__ e0,
       const T* __restrict__ e1, const T* __restrict__ e2, T* __restrict__ d0, T* __restrict__ d1,
       T* __restrict__ d2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int nseg = (c.ny + SEG - 1) / SEG;
  const int i = blockIdx.y / nseg, seg = blockIdx.y - i * nseg;
  const int comp = blockIdx.z;
  if (k >= c.nz) return;
  if (comp == 0 ? (i < 1 || i > c.nx - 1) : (i > c.nx - 1)) return;
  const size_t base = (size_t)i * plane(c) + k;
  const T* in = (comp == 0 ? e0 : comp == 1 ? e1 : e2) + base;
  T* out = (comp == 0 ? d0 : comp == 1 ? d1 : d2) + base;
  const int j0 = seg * SEG, j1 = min(j0 + SEG, c.ny);
  const size_t st = (size_t)c.nz;
  periodic_segment<T>(c.ny, j0, j1, prm->af_h, pick<T>(prm->af_rho, prm->f_rho),
                      pick<T>(1.0 / prm->r, prm->f_ir),
                      [&](int j) { return in[(size_t)j * st]; },
                      [&](int j, T v) { out[(size_t)j * st] = v; });
}

// Fused periodic factors of one (component, x plane, block of J y rows):
// (1 - aL_y) then (1 - aL_z), then u* = u^n + du. With q = 2 + 1/r and
// rho + 1/rho = q, r (q - S - S^{-1}) = (r / rho)(1 - rho S)(1 - rho S^{-1}),
// so each periodic factor is a forward recursion y_k = b_k / r + rho y_{k-1},
// a backward recursion z_k = y_k + rho z_{k+1}, and du = rho z.
//  y: one thread per z column walks its J rows (values scaled by r, so the
//     1/r of the forcing becomes one final factor). The periodic past enters
//     through a warm-up of H rows before the block (rho^H below the
//     tolerance); the periodic future through its closed form
//     z_{j0+J} = (rho y_{j0+J-1} + sum_{q<H} rho^q b_{j0+J+q}) / (1 - rho^2).
//     Results go to shared memory, rows padded by one word per 32.
//  z: one warp per row, E = nz / 32 consecutive points per lane. Each
//     recursion is a local pass, a Kogge-Stone scan of the lane carries
//     (factor rho^E per lane), and the exact periodic closure: the
//     non-periodic end value divided by (1 - rho^nz) re-enters every point
//     with weight rho^distance.
// Replaces the separate y and z kernels: reads the x factor's output and u^n
// once, writes u* once.
constexpr int YZ_THREADS = 256;
template <class T>
struct YZRows {
  static constexpr int J = sizeof(T) == 4 ? 32 : 16;
};

// E consecutive values, as 16-byte accesses when E values fill whole vectors
// (the caller's address is then 16-byte aligned)
template <class T, int E>
__device__ inline void load_run(const T* p, T (&v)[E]) {
  if constexpr (sizeof(T) == 4 && E % 4 == 0) {
#pragma unroll
    for (int t = 0; t < E; t += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + t);
      v[t] = q.x;
      v[t + 1] = q.y;
      v[t + 2] = q.z;
      v[t + 3] = q.w;
    }
  } else if constexpr (sizeof(T) == 8 && E % 2 == 0) {
#pragma unroll
    for (int t = 0; t < E; t += 2) {
      const double2 q = *reinterpret_cast<const double2*>(p + t);
      v[t] = q.x;
      v[t + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] = p[t];
  }
}
template <class T, int E>
__device__ inline void store_run(T* p, const T (&v)[E]) {
  if constexpr (sizeof(T) == 4 && E % 4 == 0) {
#pragma unroll
    for (int t = 0; t < E; t += 4)
      *reinterpret_cast<float4*>(p + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
  } else if constexpr (sizeof(T) == 8 && E % 2 == 0) {
#pragma unroll
    for (int t = 0; t < E; t += 2) *reinterpret_cast<double2*>(p + t) = make_double2(v[t], v[t + 1]);
  } else {
#pragma unroll
    for (int t = 0; t < E; ++t) p[t] = v[t];
  }
}

template <class T, int E>
__global__ void __launch_bounds__(YZ_THREADS)
k_af_yz(Consts c, const Params* __restrict__ prm, const T* __restrict__ e0,
        const T* __restrict__ e1, const T* __restrict__ e2, T* __restrict__ u,
        T* __restrict__ v, T* __restrict__ w) {
  constexpr int NZ = 32 * E;
  constexpr int LDP = NZ + NZ / 32;
  constexpr int J = YZRows<T>::J;
  __shared__ T sdu[J * LDP];
  const int ny = c.ny, ymask = c.ny - 1;   // ny is a power of two
  const int j0 = blockIdx.x * J, i = blockIdx.y, comp = blockIdx.z;
  if (comp == 0 && i < 1) return;   // u: interior faces 1 .. nx-1 only
  const size_t pb = (size_t)i * ny * NZ;
  const T* in = (comp == 0 ? e0 : comp == 1 ? e1 : e2) + pb;
  T* q = (comp == 0 ? u : comp == 1 ? v : w) + pb;
  // The recursions run on r-scaled values (y' = r y, z' = r z): the 1/r of
  // the forcing moves into one final factor rho / r per output.
  const T rho = pick<T>(prm->af_rho, prm->f_rho);
  const T rho_ir = rho * pick<T>(1.0 / prm->r, prm->f_ir);
  const int H = prm->af_h;
  const T inv_1mr2 = (T)1 / ((T)1 - rho * rho);
  // ---- y factor
  for (int k = threadIdx.x; k < NZ; k += YZ_THREADS) {
    const T* col = in + k;
    T y = 0;
    int jw = (j0 - H) & ymask;
    for (int m0 = 0; m0 < H; m0 += 8) {
      T buf[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[t] = (m0 + t < H) ? col[(size_t)((jw + t) & ymask) * NZ] : (T)0;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (m0 + t < H) y = buf[t] + rho * y;
      jw = (jw + 8) & ymask;
    }
    T yr[J];
#pragma unroll
    for (int m = 0; m < J; ++m) yr[m] = col[(size_t)(j0 + m) * NZ];
#pragma unroll
    for (int m = 0; m < J; ++m) {
      y = yr[m] + rho * y;
      yr[m] = y;
    }
    T sf = 0, pw = 1;
    jw = (j0 + J) & ymask;
    for (int m0 = 0; m0 < H; m0 += 8) {
      T buf[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[t] = (m0 + t < H) ? col[(size_t)((jw + t) & ymask) * NZ] : (T)0;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (m0 + t < H) {
          sf += pw * buf[t];
          pw *= rho;
        }
      jw = (jw + 8) & ymask;
    }
    T z = (rho * y + sf) * inv_1mr2;
    const int kp = k + (k >> 5);
#pragma unroll
    for (int m = J - 1; m >= 0; --m) {
      z = yr[m] + rho * z;
      sdu[m * LDP + kp] = rho_ir * z;
    }
  }
  __syncthreads();
  // ---- z factor, then u* = u^n + du
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T rp[E];                                   // rho^(q+1)
  rp[0] = rho;
#pragma unroll
  for (int t = 1; t < E; ++t) rp[t] = rp[t - 1] * rho;
  const T pE = rp[E - 1];                    // rho^E
  T pl = 1, pr = 1;                          // rho^(E lane), rho^(E (31 - lane))
  {
    T b = pE;
#pragma unroll
    for (int bit = 0; bit < 5; ++bit) {
      if ((lane >> bit) & 1) pl *= b;
      if (((31 - lane) >> bit) & 1) pr *= b;
      b *= b;
    }
  }
  const T rn = pl * pr * pE;                 // rho^nz
  const T inv_1mrn = (T)1 / ((T)1 - rn);
  for (int r = warp; r < J; r += YZ_THREADS / 32) {
    T* qrow = q + (size_t)(j0 + r) * NZ + lane * E;
    T un[E];
    load_run<T, E>(qrow, un);
    T x[E];
    const T* srow = sdu + r * LDP;
#pragma unroll
    for (int t = 0; t < E; ++t) {
      const int k = lane * E + t;
      x[t] = srow[k + (k >> 5)];
    }
    // forward (r-scaled): y'_k = x_k + rho y'_{k-1}
    T acc = 0;
#pragma unroll
    for (int t = 0; t < E; ++t) {
      acc = x[t] + rho * acc;
      x[t] = acc;
    }
    T Y = acc, pe = pE;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const T o = __shfl_up_sync(0xffffffffu, Y, s);
      if (lane >= s) Y += pe * o;
      pe *= pe;
    }
    const T P = __shfl_sync(0xffffffffu, Y, 31) * inv_1mrn;
    T C = __shfl_up_sync(0xffffffffu, Y, 1);
    if (lane == 0) C = 0;
    C += pl * P;
#pragma unroll
    for (int t = 0; t < E; ++t) x[t] += rp[t] * C;
    // backward: z_k = y_k + rho z_{k+1}
    acc = 0;
#pragma unroll
    for (int t = E - 1; t >= 0; --t) {
      acc = x[t] + rho * acc;
      x[t] = acc;
    }
    T Z = acc;
    pe = pE;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const T o = __shfl_down_sync(0xffffffffu, Z, s);
      if (lane + s < 32) Z += pe * o;
      pe *= pe;
    }
    const T Pz = __shfl_sync(0xffffffffu, Z, 0) * inv_1mrn;
    T C2 = __shfl_down_sync(0xffffffffu, Z, 1);
    if (lane == 31) C2 = 0;
    C2 += pr * Pz;
#pragma unroll
    for (int t = 0; t < E; ++t) un[t] += rho_ir * (x[t] + rp[E - 1 - t] * C2);
    store_run<T, E>(qrow, un);
  }
}

// z lines are contiguous: a block stages whole lines in shared memory, threads
// solve segments, and u* = u^n + du is written back.
template <class T>
__global__ void __launch_bounds__(256)
k_af_z(Consts c, const Params* __restrict__ prm, const T* __restrict__ d0,
       const T* __restrict__ d1, const T* __restrict__ d2, T* __restrict__ u, T* __restrict__ v,
       T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int nz = c.nz, ny = c.ny;
  const int ld = nz + 1;
  const int nseg = (nz + SEG - 1) / SEG;
  const int zl = blockDim.x / nseg;                    // lines per block
  const int comp = blockIdx.y;
  const int first = comp == 0 ? ny : 0;                // u: planes 1..nx-1
  const int last = c.nx * ny;                          // exclusive
  const int L0 = first + blockIdx.x * zl;
  if (L0 >= last) return;
  const int nl = min(zl, last - L0);
  const T* d = comp == 0 ? d0 : (comp == 1 ? d1 : d2);
  T* q = comp == 0 ? u : (comp == 1 ? v : w);
  const size_t base = (size_t)L0 * nz;
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    const int l = e / nz, kk = e - l * nz;
    s[l * ld + kk] = d[base + e];
  }
  __syncthreads();
  // consecutive threads take consecutive lines (row stride nz + 1: no bank conflicts)
  const int seg = threadIdx.x / zl, l = threadIdx.x - seg * zl;
  T xo[SEG];
  const int j0 = seg * SEG, j1 = min(j0 + SEG, nz);
  if (l < nl) {
    const T* line = s + l * ld;
    periodic_segment<T>(nz, j0, j1, prm->af_h, pick<T>(prm->af_rho, prm->f_rho),
                        pick<T>(1.0 / prm->r, prm->f_ir),
                        [&](int j) { return line[j]; },
                        [&](int j, T val) { xo[j - j0] = val; });
  }
  __syncthreads();
  if (l < nl) {
#pragma unroll
    for (int t = 0; t < SEG; ++t)
      if (j0 + t < j1) s[l * ld + j0 + t] = xo[t];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    const int ll = e / nz, kk = e - ll * nz;
    q[base + e] += s[ll * ld + kk];
  }
}

// FP32 periodic z factor: whole lines (plus a periodic halo) staged in shared
// memory and multiplied by the exact periodic inverse, x_j = sum_m t_|m| e_{j+m}
// (taps t from k_begin_step), truncated to |m| <= H where rho^H is below the
// FP32 rounding (all n taps when 2H + 1 >= n). No serial dependence.
template <class T>
__device__ inline void tap_range(int n, int H, int& lo, int& hi) {
  if (2 * H + 1 < n) {
    lo = H;
    hi = H;
  } else {
    lo = (n - 1) / 2;
    hi = n / 2;
  }
}

// z factor: lines contiguous; u* = u^n + du written to the velocity
constexpr int ZLC = 8;
template <class T>
__global__ void __launch_bounds__(256)
k_af_zc(Consts c, const Params* __restrict__ prm, const T* __restrict__ taps,
        const T* __restrict__ e0, const T* __restrict__ e1, const T* __restrict__ e2,
        T* __restrict__ u, T* __restrict__ v, T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int n = c.nz, ny = c.ny;
  const int comp = blockIdx.y;
  const int first = comp == 0 ? ny : 0;
  const int last = c.nx * ny;
  const int L0 = first + blockIdx.x * ZLC;
  if (L0 >= last) return;
  const int nl = min(ZLC, last - L0);
  int lo, hi;
  tap_range<T>(n, prm->af_h, lo, hi);
  const int rl = n + lo + hi;
  const T* d = comp == 0 ? e0 : (comp == 1 ? e1 : e2);
  T* qv = comp == 0 ? u : (comp == 1 ? v : w);
  const size_t base = (size_t)L0 * n;
  for (int e = threadIdx.x; e < nl * rl; e += blockDim.x) {
    const int l = e / rl, rr = e - l * rl;
    int jj = (rr - lo) % n;
    if (jj < 0) jj += n;
    s[e] = d[base + (size_t)l * n + jj];
  }
  __syncthreads();
  const int lg = __ffs(n) - 1;
  for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
    const int l = e >> lg, jj = e & (n - 1);
    const T* sl = s + l * rl + jj + lo;
    T acc = 0;
    for (int m = -lo; m <= hi; ++m) acc += taps[m < 0 ? -m : m] * sl[m];
    qv[base + e] += acc;
  }
}

// Streamed FP32 z factor: every z-row is a whole periodic line, so blocks
// stream contiguous row ranges of the RHS and of u^n through a bulk-copy
// ring (ZSTAGES slots of ZROWS rows each, mbarrier completion) and write
// u* = u^n + sum_m t_|m| e_{k+m} with the periodic wrap as an index mask.
constexpr int ZSTAGES = 6, ZROWS = 4;
template <class T>
__global__ void __launch_bounds__(256, 2)
k_af_z_pipe(Consts c, Params* __restrict__ prm, const T* __restrict__ taps,
            const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
            T* __restrict__ u, T* __restrict__ v, T* __restrict__ w, int rows_per_block) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t full[ZSTAGES];
  __shared__ T tp[2 * HMAX + 2];
  const int n = c.nz, ny = c.ny;
  const int comp = blockIdx.y;
  const int first = comp == 0 ? ny : 0;       // u: planes 1..nx-1
  const int last = c.nx * ny;
  const int r0 = first + blockIdx.x * rows_per_block;
  if (r0 >= last) return;
  const int r1 = min(r0 + rows_per_block, last);
  const int nrows = r1 - r0;
  const int nst = (nrows + ZROWS - 1) / ZROWS;
  const T* d = comp == 0 ? d0 : (comp == 1 ? d1 : d2);
  T* q = comp == 0 ? u : (comp == 1 ? v : w);
  T* ring = reinterpret_cast<T*>(smem_raw);   // [ZSTAGES][2][ZROWS][n]
  const size_t rowb = (size_t)n * sizeof(T);
  auto slot_ptr = [&](int slot) { return ring + (size_t)slot * 2 * ZROWS * n; };
  auto issue = [&](int t) {
    const int slot = t % ZSTAGES;
    const int ra = r0 + t * ZROWS;
    const int cnt = min(ZROWS, r1 - ra);
    T* st = slot_ptr(slot);
    mbar_arrive_expect_tx(&full[slot], (uint32_t)(2 * cnt * rowb));
    bulk_g2s(st, d + (size_t)ra * n, (uint32_t)(cnt * rowb), &full[slot]);
    bulk_g2s(st + (size_t)ZROWS * n, q + (size_t)ra * n, (uint32_t)(cnt * rowb), &full[slot]);
  };
  int lo, hi;
  tap_range<T>(n, prm->af_h, lo, hi);
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < ZSTAGES; ++sl) mbar_init(&full[sl], 1);
    fence_mbar_init();
  }
  for (int m = threadIdx.x; m <= max(lo, hi); m += blockDim.x) tp[m] = taps[m];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 0; t < ZSTAGES && t < nst; ++t) issue(t);
  const int mask = n - 1, lg = __ffs(n) - 1;
  for (int t = 0; t < nst; ++t) {
    const bool ok = mbar_wait(&full[t % ZSTAGES], (uint32_t)((t / ZSTAGES) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&prm->error, ERR_TIMEOUT);
        for (int tt = t; tt < nst && tt < t + ZSTAGES; ++tt)
          (void)mbar_wait(&full[tt % ZSTAGES], (uint32_t)((tt / ZSTAGES) & 1));
      }
      return;
    }
    const T* st = slot_ptr(t % ZSTAGES);
    const int ra = r0 + t * ZROWS;
    const int cnt = min(ZROWS, r1 - ra);
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
      const int l = e >> lg, k = e & mask;
      const T* dl = st + (size_t)l * n;
      T acc = tp[0] * dl[k];
      for (int m = 1; m <= lo && m <= hi; ++m) acc += tp[m] * (dl[(k + m) & mask] + dl[(k - m) & mask]);
      if (hi > lo) acc += tp[hi] * dl[(k + hi) & mask];
      q[(size_t)ra * n + e] = st[(size_t)ZROWS * n + e] + acc;
    }
    __syncthreads();
    if (threadIdx.x == 0 && t + ZSTAGES < nst) issue(t + ZSTAGES);
  }
}

// ---------------------------------------------------------------- mass fix + divergence (A7)
// Q_in, Q_out over the inflow/outflow faces (FP64, fixed summation order);
// the shift (Q_in - Q_out) / (Ly Lz) goes onto the outflow face.
// reduce the outflow kernel's per-block flux partials (fixed order)
__global__ void k_mass(Consts c, Params* prm, const double* __restrict__ qpart, int nb) {
  __shared__ double scratch[32];
  double qi = 0.0, qo = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    qi += qpart[2 * b];
    qo += qpart[2 * b + 1];
  }
  qi = block_sum(qi, scratch);
  __syncthreads();
  qo = block_sum(qo, scratch);
  if (threadIdx.x == 0) {
    const double h2 = c.h * c.h;
    prm->q_in = qi * h2;
    prm->q_out = qo * h2;
    prm->mass_shift = (qi - qo) * h2 / (c.ly * c.lz);
    prm->f_mass_shift = (float)prm->mass_shift;
  }
}

template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_div(Consts c, const Params* __restrict__ prm, T* __restrict__ u, const T* __restrict__ v,
      const T* __restrict__ w, T* __restrict__ phi, int initial) {
  const int k = blockIdx.x * TK + threadIdx.x;
  const int j = blockIdx.y * TJ + threadIdx.y;
  if (k >= c.nz || j >= c.ny) return;
  const int ny = c.ny, nz = c.nz, nx = c.nx;
  const int jp = j == ny - 1 ? 0 : j + 1, kp = k == nz - 1 ? 0 : k + 1;
  const size_t P = plane(c);
  const T shift = initial ? (T)0 : pick<T>(prm->mass_shift, prm->f_mass_shift);
  const T sc = initial ? pick<T>(c.inv_h, c.f_inv_h) : pick<T>(c.inv_h / prm->dt, prm->f_sc_div);
  const int i0 = blockIdx.z * XCHUNK, i1 = min(i0 + XCHUNK, nx);
  for (int i = i0; i < i1; ++i) {
    const size_t id = ((size_t)i * ny + j) * nz + k;
    T ue = u[id + P];
    if (i == nx - 1) {
      ue += shift;
      u[id + P] = ue;
    }
    const T dv = (ue - u[id]) + (v[((size_t)i * ny + jp) * nz + k] - v[id]) +
                 (w[((size_t)i * ny + j) * nz + kp] - w[id]);
    phi[id] = dv * sc;
  }
}

// ---------------------------------------------------------------- projection (A9)
// u^{n+1} = u** - dt G phi (interior faces), p^{n+1} = p^n + phi - (nu dt / 2) L phi,
// written to the other velocity buffer; per-block maxima of the cell speed
// |u_c| + |v_c| + |w_c| of the new velocity feed the next CFL step.
template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_project(Consts c, const Params* __restrict__ prm, const T* __restrict__ ua,
          const T* __restrict__ va, const T* __restrict__ wa, T* __restrict__ ub,
          T* __restrict__ vb, T* __restrict__ wb, const T* __restrict__ phi_a, const T* __restrict__ phi_b,
          T* __restrict__ p, double* __restrict__ partial, int initial) {
  // phi = phi_a (+ phi_b: the mixed solve's predictor and correction, summed here)
  auto phiv = [&](size_t q) { return phi_b ? phi_a[q] + phi_b[q] : phi_a[q]; };
  const int k = blockIdx.x * TK + threadIdx.x;
  const int j = blockIdx.y * TJ + threadIdx.y;
  const bool act = (k < c.nz && j < c.ny);
  const int ny = c.ny, nz = c.nz, nx = c.nx;
  const size_t P = plane(c);
  T smaxT = 0;
  if (act) {
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
    const T gdt = initial ? pick<T>(c.inv_h, c.f_inv_h) : pick<T>(prm->dt * c.inv_h, prm->f_gdt);
    const T hnu = initial ? (T)0 : pick<T>(0.5 * c.nu * prm->dt * c.inv_h * c.inv_h, prm->f_hnu);
    auto at = [&](int i, int jj, int kk) { return ((size_t)i * ny + jj) * nz + kk; };
    auto unew = [&](int i) -> T {  // new u on face i at (j, k)
      const size_t id = at(i, j, k);
      if (i >= 1 && i <= nx - 1) return ua[id] - gdt * (phiv(id) - phiv(id - P));
      return ua[id];
    };
    const int i0 = blockIdx.z * XCHUNK, i1 = min(i0 + XCHUNK, nx + 1);
    for (int i = i0; i < i1; ++i) {
      const size_t id = at(i, j, k);
      const T un = unew(i);
      ub[id] = un;
      if (i == nx) {
        vb[id] = va[id];
        wb[id] = wa[id];
        continue;
      }
      const T ph = phiv(id);
      const T vn = va[id] - gdt * (ph - phiv(at(i, jm, k)));
      const T wn = wa[id] - gdt * (ph - phiv(at(i, j, km)));
      vb[id] = vn;
      wb[id] = wn;
      if (!initial) {
        const T pxm = i == 0 ? ph : phiv(id - P);
        const T pxp = i == nx - 1 ? ph : phiv(id + P);
        const T lap = pxm + pxp + phiv(at(i, jm, k)) + phiv(at(i, jp, k)) + phiv(at(i, j, km)) +
                      phiv(at(i, j, kp)) - (T)6 * ph;
        p[id] += ph - hnu * lap;
      }
      const T un1 = unew(i + 1);
      const T vn1 = va[at(i, jp, k)] - gdt * (phiv(at(i, jp, k)) - ph);
      const T wn1 = wa[at(i, j, kp)] - gdt * (phiv(at(i, j, kp)) - ph);
      T sp = fabs((T)0.5 * (un + un1)) + fabs((T)0.5 * (vn + vn1)) + fabs((T)0.5 * (wn + wn1));
      if (!isfinite(sp)) sp = (T)INFINITY;
      smaxT = fmax(smaxT, sp);
    }
  }
  // flatten the 2-D block for the reduction (in T: a max is exact)
  const int tid = threadIdx.y * TK + threadIdx.x;
  T v = smaxT;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ T wmax[TK * TJ / 32];
  if ((tid & 31) == 0) wmax[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    T m = 0;
    for (int q = 0; q < TK * TJ / 32; ++q) m = fmax(m, wmax[q]);
    partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = (double)m;
  }
}

// Vector forms of the divergence and the projection: a thread owns a run of
// E = 16 / sizeof(T) consecutive z points of one row and walks x planes, so
// every field access is a 16-byte load or store (single values at the run's
// two z edges); the projection keeps phi of planes i-1, i, i+1 and the new u
// of the next face in registers. Block: TJ rows x (nz / E) runs = 256 threads.
template <class T>
struct RunTile {
  static constexpr int E = 16 / sizeof(T);
  static constexpr int THREADS = 256;
};
// rows per block of the run kernels, 0 when the shape does not fit them
template <class T>
int run_rows(const Consts& c) {
  const int runs = c.nz / RunTile<T>::E;
  if (runs < 1 || runs > RunTile<T>::THREADS || RunTile<T>::THREADS % runs) return 0;
  const int tj = RunTile<T>::THREADS / runs;
  return c.ny % tj == 0 ? tj : 0;
}
constexpr int RUN_XCH = 16;   // x planes per block of the run kernels

template <class T>
__global__ void __launch_bounds__(256)
k_div_vec(Consts c, const Params* __restrict__ prm, T* __restrict__ u, const T* __restrict__ v,
          const T* __restrict__ w, T* __restrict__ phi, int initial) {
  constexpr int E = RunTile<T>::E;
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int runs = nz / E;
  const int tj = RunTile<T>::THREADS / runs;
  const int r = threadIdx.x / runs, k0 = (threadIdx.x - r * runs) * E;
  const int j = blockIdx.x * tj + r;
  const int jp = (j + 1) & (ny - 1), kpE = (k0 + E) & (nz - 1);
  const size_t P = plane(c);
  const T shift = initial ? (T)0 : pick<T>(prm->mass_shift, prm->f_mass_shift);
  const T sc = initial ? pick<T>(c.inv_h, c.f_inv_h) : pick<T>(c.inv_h / prm->dt, prm->f_sc_div);
  const int i0 = blockIdx.y * RUN_XCH, i1 = min(i0 + RUN_XCH, nx);
  if (i0 >= i1) return;
  T uw[E];
  ldg_run<T, E>(u + ((size_t)i0 * ny + j) * nz + k0, uw);
  for (int i = i0; i < i1; ++i) {
    const size_t id = ((size_t)i * ny + j) * nz + k0;
    T ue[E], vv[E], vn[E], ww[E], dv[E];
    ldg_run<T, E>(u + id + P, ue);
    ldg_run<T, E>(v + id, vv);
    ldg_run<T, E>(v + ((size_t)i * ny + jp) * nz + k0, vn);
    ldg_run<T, E>(w + id, ww);
    const T w_r = w[((size_t)i * ny + j) * nz + kpE];
    if (i == nx - 1) {
#pragma unroll
      for (int e = 0; e < E; ++e) ue[e] += shift;
      stg_run<T, E>(u + id + P, ue);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T wp = e == E - 1 ? w_r : ww[e + 1];
      dv[e] = ((ue[e] - uw[e]) + (vn[e] - vv[e]) + (wp - ww[e])) * sc;
      uw[e] = ue[e];
    }
    stg_run<T, E>(phi + id, dv);
  }
}

// TWO: 0 phi alone; 1 phi + phi_b (FP32); 2 phi + phi_b (bfloat16) -- the
// mixed solve's predictor and correction, summed as they are read
// two blocks per SM: the register budget of three made every variant spill
// (0.262 against 0.207 ms for the mixed instance)
template <class T, int TWO>
__global__ void __launch_bounds__(256, 2)
k_project_vec(Consts c, const Params* __restrict__ prm, const T* __restrict__ ua,
              const T* __restrict__ va, const T* __restrict__ wa, T* __restrict__ ub,
              T* __restrict__ vb, T* __restrict__ wb, const T* __restrict__ phi, const void* __restrict__ phi_b,
              T* __restrict__ p, double* __restrict__ partial, int initial) {
  constexpr int E = RunTile<T>::E;
  const T* pb = static_cast<const T*>(phi_b);
  const __nv_bfloat16* pb16 = static_cast<const __nv_bfloat16*>(phi_b);
  auto ldg_phi = [&](size_t q, T (&v)[E]) {
    ldg_run<T, E>(phi + q, v);
    if constexpr (TWO == 1) {
      T t[E];
      ldg_run<T, E>(pb + q, t);
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = v[e] + t[e];
    } else if constexpr (TWO == 2) {
      static_assert(E == 4 && sizeof(T) == 4, "bfloat16 correction with FP32 runs of four");
      const uint2 r = *reinterpret_cast<const uint2*>(pb16 + q);
      v[0] += __uint_as_float(r.x << 16);
      v[1] += __uint_as_float(r.x & 0xFFFF0000u);
      v[2] += __uint_as_float(r.y << 16);
      v[3] += __uint_as_float(r.y & 0xFFFF0000u);
    }
  };
  auto phi1 = [&](size_t q) {
    if constexpr (TWO == 1) return phi[q] + pb[q];
    else if constexpr (TWO == 2) return phi[q] + (T)__bfloat162float(pb16[q]);
    else return phi[q];
  };
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int runs = nz / E;
  const int tj = RunTile<T>::THREADS / runs;
  const int tid = threadIdx.x;
  const int r = tid / runs, k0 = (tid - r * runs) * E;
  const int j = blockIdx.x * tj + r;
  const int jm = (j - 1) & (ny - 1), jp = (j + 1) & (ny - 1);
  const int km1 = (k0 - 1) & (nz - 1), kpE = (k0 + E) & (nz - 1);
  auto at = [&](int i, int jj, int kk) { return ((size_t)i * ny + jj) * nz + kk; };
  const T gdt = initial ? pick<T>(c.inv_h, c.f_inv_h) : pick<T>(prm->dt * c.inv_h, prm->f_gdt);
  const T hnu = initial ? (T)0 : pick<T>(0.5 * c.nu * prm->dt * c.inv_h * c.inv_h, prm->f_hnu);
  const int i0 = blockIdx.y * RUN_XCH, i1 = min(i0 + RUN_XCH, nx + 1);
  T smax = 0;
  T phm[E], ph[E], php[E], un[E], un1[E];
#pragma unroll
  for (int e = 0; e < E; ++e) phm[e] = ph[e] = (T)0;
  if (i0 >= 1 && i0 - 1 <= nx - 1) ldg_phi(at(i0 - 1, j, k0), phm);
  if (i0 <= nx - 1) ldg_phi(at(i0, j, k0), ph);
  ldg_run<T, E>(ua + at(i0, j, k0), un);
  if (i0 >= 1 && i0 <= nx - 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) un[e] -= gdt * (ph[e] - phm[e]);
  }
  for (int i = i0; i < i1; ++i) {
    const size_t id = at(i, j, k0);
    if (i == nx) {   // outflow face and the ghost planes of v, w: copies
      T t[E];
      stg_run<T, E>(ub + id, un);
      ldg_run<T, E>(va + id, t);
      stg_run<T, E>(vb + id, t);
      ldg_run<T, E>(wa + id, t);
      stg_run<T, E>(wb + id, t);
      break;
    }
    // next plane: phi (Neumann image at the last plane) and the new u of face i+1
    if (i + 1 <= nx - 1) {
      ldg_phi(id + plane(c), php);
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) php[e] = ph[e];
    }
    ldg_run<T, E>(ua + id + plane(c), un1);
    if (i + 1 <= nx - 1) {
#pragma unroll
      for (int e = 0; e < E; ++e) un1[e] -= gdt * (php[e] - ph[e]);
    }
    T vv[E], vjp[E], ww[E], pjm[E], pjp[E], pp[E];
    ldg_run<T, E>(va + id, vv);
    ldg_run<T, E>(va + at(i, jp, k0), vjp);
    ldg_run<T, E>(wa + id, ww);
    ldg_phi(at(i, jm, k0), pjm);
    ldg_phi(at(i, jp, k0), pjp);
    const T w_r = wa[at(i, j, kpE)];
    const T ph_l = phi1(at(i, j, km1)), ph_r = phi1(at(i, j, kpE));
    if (!initial) ldg_run<T, E>(p + id, pp);
    stg_run<T, E>(ub + id, un);
    T vo[E], wo[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T pl = e == 0 ? ph_l : ph[e - 1], pr = e == E - 1 ? ph_r : ph[e + 1];
      const T wr = e == E - 1 ? w_r : ww[e + 1];
      const T vn = vv[e] - gdt * (ph[e] - pjm[e]);
      const T wn = ww[e] - gdt * (ph[e] - pl);
      vo[e] = vn;
      wo[e] = wn;
      const T vn1 = vjp[e] - gdt * (pjp[e] - ph[e]);
      const T wn1 = wr - gdt * (pr - ph[e]);
      if (!initial) {
        const T pxm = i == 0 ? ph[e] : phm[e];
        const T lap = pxm + php[e] + pjm[e] + pjp[e] + pl + pr - (T)6 * ph[e];
        pp[e] += ph[e] - hnu * lap;
      }
      T sp = fabs((T)0.5 * (un[e] + un1[e])) + fabs((T)0.5 * (vn + vn1)) +
             fabs((T)0.5 * (wn + wn1));
      if (!isfinite(sp)) sp = (T)INFINITY;
      smax = fmax(smax, sp);
    }
    stg_run<T, E>(vb + id, vo);
    stg_run<T, E>(wb + id, wo);
    if (!initial) stg_run<T, E>(p + id, pp);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      phm[e] = ph[e];
      ph[e] = php[e];
      un[e] = un1[e];
    }
  }
  // block maximum (in T: a max is exact)
  T vmax = smax;
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  __shared__ T wmax[RunTile<T>::THREADS / 32];
  if ((tid & 31) == 0) wmax[tid >> 5] = vmax;
  __syncthreads();
  if (tid == 0) {
    T m = 0;
    for (int q = 0; q < RunTile<T>::THREADS / 32; ++q) m = fmax(m, wmax[q]);
    partial[blockIdx.y * gridDim.x + blockIdx.x] = (double)m;
  }
}

// ---------------------------------------------------------------- diagnostics
// out[0] += kinetic energy, out[1] = max |div u| (atomics; diagnostics only)
template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_stats(Consts c, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
        double* out) {
  const int k = blockIdx.x * TK + threadIdx.x;
  const int j = blockIdx.y * TJ + threadIdx.y;
  double ke = 0.0, dmax = 0.0;
  if (k < c.nz && j < c.ny) {
    const int ny = c.ny, nz = c.nz, nx = c.nx;
    const int jp = j == ny - 1 ? 0 : j + 1, kp = k == nz - 1 ? 0 : k + 1;
    const size_t P = plane(c);
    const int i0 = blockIdx.z * XCHUNK, i1 = min(i0 + XCHUNK, nx + 1);
    for (int i = i0; i < i1; ++i) {
      const size_t id = ((size_t)i * ny + j) * nz + k;
      const double uu = u[id];
      ke += 0.5 * uu * uu;
      if (i < nx) {
        const double vv = v[id], ww = w[id];
        ke += 0.5 * (vv * vv + ww * ww);
        const double dv = ((double)u[id + P] - uu) + ((double)v[((size_t)i * ny + jp) * nz + k] - vv) +
                          ((double)w[((size_t)i * ny + j) * nz + kp] - ww);
        dmax = fmax(dmax, fabs(dv) * c.inv_h);
      }
    }
  }
  ke = warp_sum(ke);
  dmax = warp_max(dmax);
  if (((threadIdx.y * TK + threadIdx.x) & 31) == 0) {
    atomicAdd(&out[0], ke * c.h * c.h * c.h);
    atomic_max_nonneg(&out[1], dmax);
  }
}

// ---------------------------------------------------------------- launchers
static dim3 grid3(const Consts& c, int planes) {
  return dim3((c.nz + TK - 1) / TK, (c.ny + TJ - 1) / TJ, (planes + XCHUNK - 1) / XCHUNK);
}

// ---------------------------------------------------------------- prescribed inflow
// plane q of the inflow block: 0..2 pending u, v, w; 3, 4 current v, w;
// 5..7 increments u, v, w
template <class T>
static T* inflow_plane(const Consts& c, const Fields<T>& f, int q) {
  return f.inflow ? f.inflow + (size_t)q * c.ny * c.nz : nullptr;
}
template <class T>
static const T* inflow_cur_v(const Consts& c, const Fields<T>& f) { return inflow_plane(c, f, 3); }
template <class T>
static const T* inflow_cur_w(const Consts& c, const Fields<T>& f) { return inflow_plane(c, f, 4); }
template <class T>
static const T* inflow_inc(const Consts& c, const Fields<T>& f) { return inflow_plane(c, f, 5); }

// mean of the pending u plane, FP64, fixed order (one block)
template <class T>
__global__ void k_inflow_mean(Consts c, const T* __restrict__ pu, double* __restrict__ mean) {
  __shared__ double scratch[32];
  const int P = c.ny * c.nz;
  double s = 0.0;
  for (int q = threadIdx.x; q < P; q += blockDim.x) s += (double)pu[q];
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) *mean = s / P;
}

// the new inflow time level: u_in = pending u - mean + U on face 0, the
// boundary increments for the x factor, and the current v, w planes
template <class T>
__global__ void k_inflow_advance(Consts c, T* __restrict__ blk, const double* __restrict__ mean,
                                 T* __restrict__ u) {
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  T* pu = blk;
  T* pv = blk + P;
  T* pw = blk + 2 * (size_t)P;
  T* cv = blk + 3 * (size_t)P;
  T* cw = blk + 4 * (size_t)P;
  T* iu = blk + 5 * (size_t)P;
  T* iv = blk + 6 * (size_t)P;
  T* iw = blk + 7 * (size_t)P;
  const T un = (T)((double)pu[jk] - *mean + c.u_in);
  iu[jk] = un - u[jk];
  u[jk] = un;
  const T vn = pv[jk], wn = pw[jk];
  iv[jk] = vn - cv[jk];
  iw[jk] = wn - cw[jk];
  cv[jk] = vn;
  cw[jk] = wn;
}

template <class T>
void launch_inflow(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  if (!f.inflow) return;
  const int P = c.ny * c.nz;
  k_inflow_mean<T><<<1, 1024, 0, s>>>(c, f.inflow, f.inflow_mean);
  k_inflow_advance<T><<<(P + 255) / 256, 256, 0, s>>>(c, f.inflow, f.inflow_mean, f.u[cur]);
}

template <class T>
void launch_begin_step(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const double tol = sizeof(T) == 8 ? 1e-17 : 1e-9;
  k_begin_step<<<1, 1024, 0, s>>>(c, f.prm, f.partial, f.n_partial, tol, hmax_of<T>());
}

template <class T>
void launch_af_tables(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const int n = table_entries(c);
  k_af_tables<<<(n + TAB_THREADS - 1) / TAB_THREADS, TAB_THREADS, 0, s>>>(c, f.prm, f.ipt, f.iptf,
                                                                          f.taps, f.tapsf);
}

template <class T>
static size_t rhs_stage_bytes(const Consts& c, int tjr) {
  return (size_t)(3 * (tjr + 2) + (tjr + 1) + 3 * tjr) * c.nz * sizeof(T);
}

template <class T>
void launch_rhs(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  {
    using RV = RhsVec<T>;
    const int threads = RV::TJ * (c.nz / RV::E);
    const size_t sh = (size_t)RV::STAGES * RV::ROWS * c.nz * sizeof(T);
    if (threads % 32 == 0 && threads <= 256 && c.ny % RV::TJ == 0 && sh <= 200 * 1024) {
      const int XR = c.rhs_planes;
      k_rhs_vec<T><<<dim3(c.ny / RV::TJ, (c.nx + XR - 1) / XR), threads, sh, s>>>(
          c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.p, f.n[0], f.n[1], f.n[2], f.d[0], f.d[1],
          f.d[2], XR, inflow_cur_v(c, f), inflow_cur_w(c, f));
      return;
    }
  }
  constexpr int TJR = sizeof(T) == 4 ? 4 : 2;
  const size_t stage = rhs_stage_bytes<T>(c, TJR);
  const int rs = (int)std::min<size_t>(std::min(RSTAGES_MAX, c.rhs_stages), (size_t)(210 * 1024) / stage);
  if (rs >= 4 && c.ny % TJR == 0 && (c.nz * sizeof(T)) % 16 == 0) {
    const int XR = c.rhs_planes;
    k_rhs_pipe<T, TJR><<<dim3(c.ny / TJR, (c.nx + XR - 1) / XR), RTHREADS, rs * stage, s>>>(
        c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.p, f.n[0], f.n[1], f.n[2], f.d[0], f.d[1],
        f.d[2], XR, rs, inflow_cur_v(c, f), inflow_cur_w(c, f));
    return;
  }
  k_rhs<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                        f.p, f.n[0], f.n[1], f.n[2], f.d[0],
                                                        f.d[1], f.d[2], inflow_cur_v(c, f),
                                                        inflow_cur_w(c, f));
}

int outflow_blocks(const Consts& c) { return (c.ny * c.nz + OUT_THREADS - 1) / OUT_THREADS; }

// one case of the ensemble's explicit stage (k_rhs_cases)
template <class T>
RhsCase<T> rhs_case(const Consts& c, const Fields<T>& f, int cur) {
  RhsCase<T> e{};
  e.c = c;
  e.prm = f.prm;
  e.u = f.u[cur];
  e.v = f.v[cur];
  e.w = f.w[cur];
  e.p = f.p;
  e.n0 = f.n[0];
  e.n1 = f.n[1];
  e.n2 = f.n[2];
  e.d0 = f.d[0];
  e.d1 = f.d[1];
  e.d2 = f.d[2];
  e.vin = inflow_cur_v(c, f);
  e.win = inflow_cur_w(c, f);
  const dim3 g = grid3(c, c.nx + 1);
  e.gx = (int)g.x;
  e.gy = (int)g.y;
  e.gz = (int)g.z;
  return e;
}

template <class T>
void launch_rhs_cases(const RhsCase<T>* table, int ncases, int total, int blocks, cudaStream_t s) {
  k_rhs_cases<T><<<blocks, dim3(TK, TJ), 0, s>>>(table, ncases, total);
}

template <class T>
void launch_outflow(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  k_outflow<T><<<outflow_blocks(c), OUT_THREADS, 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                         f.dout[0], f.dout[1], f.dout[2], f.qpart);
}

template <class T>
void launch_af_x(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  const int P = c.ny * c.nz;
  {
    const T* tab;
    if constexpr (sizeof(T) == 8) tab = (const T*)f.ipt; else tab = (const T*)f.iptf;
    // afx_planes selects the x segment: 16 or 24 planes per thread in registers,
    if (c.afx_planes == 16 || c.afx_planes == 24) {
      const int xv = c.afx_planes;
      const dim3 grid((P + 255) / 256, (c.nx + xv - 1) / xv, 3);
      if (xv == 16)
        k_af_xv<T, 16><<<grid, 256, 0, s>>>(c, f.prm, tab, f.d[0], f.d[1], f.d[2], f.e[0], f.e[1],
                                            f.e[2], f.dout[0], f.dout[1], f.dout[2],
                                            inflow_inc(c, f));
      else
        k_af_xv<T, 24><<<grid, 256, 0, s>>>(c, f.prm, tab, f.d[0], f.d[1], f.d[2], f.e[0], f.e[1],
                                            f.e[2], f.dout[0], f.dout[1], f.dout[2],
                                            inflow_inc(c, f));
      return;
    }
    // otherwise segments of 32 or 64 planes staged in shared memory by warps
    if (c.afx_planes <= 40) {
      k_af_xr<T, 32><<<dim3((P + 31) / 32, (c.nx + 31) / 32, 3), 32, 0, s>>>(
          c, f.prm, tab, f.d[0], f.d[1], f.d[2], f.e[0], f.e[1], f.e[2], f.dout[0], f.dout[1],
          f.dout[2], inflow_inc(c, f));
    } else {
      k_af_xr<T, 64><<<dim3((P + 31) / 32, (c.nx + 63) / 64, 3), 32, 0, s>>>(
          c, f.prm, tab, f.d[0], f.d[1], f.d[2], f.e[0], f.e[1], f.e[2], f.dout[0], f.dout[1],
          f.dout[2], inflow_inc(c, f));
    }
    (void)cur;
  }
}

template <class T>
void launch_af_y(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  const int nseg = (c.ny + SEG - 1) / SEG;
  k_af_y<T><<<dim3((c.nz + 127) / 128, c.nx * nseg, 3), 128, 0, s>>>(c, f.prm, f.e[0], f.e[1],
                                                                       f.e[2], f.d[0], f.d[1], f.d[2]);
  (void)cur;
}

static int af_z_lines(const Consts& c) { return 256 / ((c.nz + SEG - 1) / SEG); }

template <class T>
void launch_af_z(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if ((c.nz * sizeof(T)) % 16 == 0) {
      const int rpb = 512;
      const size_t sh = (size_t)ZSTAGES * 2 * ZROWS * c.nz * sizeof(T);
      k_af_z_pipe<T><<<dim3((c.nx * c.ny + rpb - 1) / rpb, 3), 256, sh, s>>>(
          c, f.prm, (const T*)f.tapsf + c.ny, f.d[0], f.d[1], f.d[2], f.u[cur], f.v[cur], f.w[cur],
          rpb);
      return;
    }
    const int halo = HMAX < c.nz / 2 ? HMAX : c.nz / 2;
    const size_t sh = (size_t)ZLC * (c.nz + 2 * halo) * sizeof(T);
    k_af_zc<T><<<dim3((c.nx * c.ny + ZLC - 1) / ZLC, 3), 256, sh, s>>>(
        c, f.prm, (const T*)f.tapsf + c.ny, f.d[0], f.d[1], f.d[2], f.u[cur], f.v[cur], f.w[cur]);
    return;
  }
  const int zl = af_z_lines(c);
  const size_t shz = (size_t)zl * (c.nz + 1) * sizeof(T);
  k_af_z<T><<<dim3((c.nx * c.ny + zl - 1) / zl, 3), 256, shz, s>>>(
      c, f.prm, f.d[0], f.d[1], f.d[2], f.u[cur], f.v[cur], f.w[cur]);
}

// fused y-z factors for nz = 32 E with E in {1, 2, 4, 8} and ny a multiple of
// the row block; false when the shape needs the separate kernels
template <class T>
bool launch_af_yz(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  constexpr int J = YZRows<T>::J;
  if (c.ny % J != 0) return false;
  const dim3 grid(c.ny / J, c.nx, 3);
#define YZ_CASE(EE)                                                                               \
  case 32 * EE:                                                                                   \
    k_af_yz<T, EE><<<grid, YZ_THREADS, 0, s>>>(c, f.prm, f.e[0], f.e[1], f.e[2], f.u[cur],       \
                                              f.v[cur], f.w[cur]);                               \
    return true;
  switch (c.nz) {
    YZ_CASE(1)
    YZ_CASE(2)
    YZ_CASE(4)
    YZ_CASE(8)
    default: return false;
  }
#undef YZ_CASE
}

template <class T>
void launch_af(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  launch_af_x(c, f, cur, s);
  if (launch_af_yz(c, f, cur, s)) return;
  launch_af_y(c, f, cur, s);
  launch_af_z(c, f, cur, s);
}

template <class T>
void launch_mass(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  k_mass<<<1, 1024, 0, s>>>(c, f.prm, f.qpart, outflow_blocks(c));
  (void)cur;
}

template <class T>
void launch_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  if (const int tj = run_rows<T>(c)) {
    k_div_vec<T><<<dim3(c.ny / tj, (c.nx + RUN_XCH - 1) / RUN_XCH), RunTile<T>::THREADS, 0, s>>>(
        c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.phi, initial ? 1 : 0);
    return;
  }
  k_div<T><<<grid3(c, c.nx), dim3(TK, TJ), 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.phi,
                                                    initial ? 1 : 0);
}

template <class T>
void launch_mass_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  if (!initial) launch_mass(c, f, cur, s);
  launch_div(c, f, cur, initial, s);
}

// phi = phi_a + phi_b when phi_b is given (the mixed solve's predictor and
// correction), phi_a = f.phi when not given
template <class T>
void launch_project_only(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s,
                         const T* phi_a, const T* phi_b, const void* phi_b16) {
  if (!phi_a) phi_a = f.phi;
  if (const int tj = run_rows<T>(c)) {
    const dim3 grid(c.ny / tj, (c.nx + 1 + RUN_XCH - 1) / RUN_XCH);
    const int ini = initial ? 1 : 0;
    if constexpr (sizeof(T) == 4 && RunTile<T>::E == 4) {
      if (phi_b16) {
        k_project_vec<T, 2><<<grid, RunTile<T>::THREADS, 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                                f.u[cur ^ 1], f.v[cur ^ 1], f.w[cur ^ 1],
                                                                phi_a, phi_b16, f.p, f.partial, ini);
        return;
      }
    }
    if (phi_b)
      k_project_vec<T, 1><<<grid, RunTile<T>::THREADS, 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                              f.u[cur ^ 1], f.v[cur ^ 1], f.w[cur ^ 1],
                                                              phi_a, phi_b, f.p, f.partial, ini);
    else
      k_project_vec<T, 0><<<grid, RunTile<T>::THREADS, 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                              f.u[cur ^ 1], f.v[cur ^ 1], f.w[cur ^ 1],
                                                              phi_a, nullptr, f.p, f.partial, ini);
    return;
  }
  k_project<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(
      c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.u[cur ^ 1], f.v[cur ^ 1], f.w[cur ^ 1], phi_a, phi_b, f.p,
      f.partial, initial ? 1 : 0);
}

template <class T>
void launch_project(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s,
                    const T* phi_a, const T* phi_b, const void* phi_b16) {
  launch_project_only(c, f, cur, initial, s, phi_a, phi_b, phi_b16);
  if (!initial) k_end_step<<<1, 1, 0, s>>>(f.prm);
}

template <class T>
void launch_stats(const Consts& c, const Fields<T>& f, int cur, double* out, cudaStream_t s) {
  k_stats<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(c, f.u[cur], f.v[cur], f.w[cur], out);
}

void fluid_set_attributes() {
  cudaFuncSetAttribute(k_rhs_pipe<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  cudaFuncSetAttribute(k_rhs_vec<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_rhs_vec<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_rhs_pipe<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  cudaFuncSetAttribute(k_af_zc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_z_pipe<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_z<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_z<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// blocks of the projection launch (one CFL partial each)
template <class T>
int partial_count(const Consts& c) {
  if (const int tj = run_rows<T>(c)) return c.ny / tj * ((c.nx + 1 + RUN_XCH - 1) / RUN_XCH);
  const dim3 g = grid3(c, c.nx + 1);
  return (int)(g.x * g.y * g.z);
}
template int partial_count<float>(const Consts&);
template int partial_count<double>(const Consts&);

#define INST(T)                                                                                \
  template void launch_begin_step<T>(const Consts&, const Fields<T>&, cudaStream_t);           \
  template void launch_rhs<T>(const Consts&, const Fields<T>&, int, cudaStream_t);             \
  template RhsCase<T> rhs_case<T>(const Consts&, const Fields<T>&, int);                       \
  template void launch_rhs_cases<T>(const RhsCase<T>*, int, int, int, cudaStream_t);          \
  template void launch_af_tables<T>(const Consts&, const Fields<T>&, cudaStream_t);             \
  template void launch_inflow<T>(const Consts&, const Fields<T>&, int, cudaStream_t);           \
  template void launch_outflow<T>(const Consts&, const Fields<T>&, int, cudaStream_t);         \
  template void launch_af<T>(const Consts&, const Fields<T>&, int, cudaStream_t);              \
  template void launch_af_x<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_af_y<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_af_z<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template bool launch_af_yz<T>(const Consts&, const Fields<T>&, int, cudaStream_t);           \
  template void launch_mass<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_div<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t);       \
  template void launch_project_only<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t, const T*, \
                                       const T*, const void*);                                     \
  template void launch_mass_div<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t);  \
  template void launch_project<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t, const T*, \
                                  const T*, const void*);                                          \
  template void launch_stats<T>(const Consts&, const Fields<T>&, int, double*, cudaStream_t);
INST(double)
INST(float)

}  // namespace ibm
