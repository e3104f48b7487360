// Fluid kernels of one fractional step (Sec. II.B): per-step parameters,
// explicit right-hand side (AB2 advection, explicit half of Crank--Nicolson,
// pressure gradient), convective outflow (Sec. II.A), the three implicit
// factors of the approximate factorisation, the mass fix and divergence, and
// the projection with the pressure update.
//
// Layout: x slowest, z fastest; u, v, w have nx + 1 planes (u: faces
// 0..nx; v, w: cells 0..nx-1 plus the outflow ghost plane nx), p and phi nx.
#include <cmath>

#include "solver.h"

namespace ibm {

constexpr int TK = 32;       // threads along z in 3-D kernels
constexpr int TJ = 8;        // threads along y
constexpr int XCHUNK = 8;    // x planes per block in 3-D kernels

// ---------------------------------------------------------------- parameters
// dt (fixed or CFL), AB2 weights, implicit diffusion number, sub-steps.
__global__ void k_begin_step(Consts c, Params* prm, const double* __restrict__ partial,
                             int n_partial) {
  __shared__ double scratch[32];
  double m = 0.0;
  for (int b = threadIdx.x; b < n_partial; b += blockDim.x) m = fmax(m, partial[b]);
  m = block_max(m, scratch);
  if (threadIdx.x != 0) return;
  Params p = *prm;
  p.speed_max = m;
  p.slip_max = 0.0;
  double dt = p.dt_fixed > 0.0 ? p.dt_fixed : p.cfl * c.h / m;
  if (!isfinite(m) || !(dt > 0.0) || !isfinite(dt)) {
    p.error |= ERR_NONFINITE;
    dt = p.dt_fixed > 0.0 ? p.dt_fixed : 0.0;
  }
  if (p.first) {
    p.alpha = 1.0;
    p.beta = 0.0;
  } else {
    p.alpha = 1.0 + dt / (2.0 * p.dt_old);
    p.beta = -dt / (2.0 * p.dt_old);
  }
  p.dt = dt;
  p.r = c.nu * dt / (2.0 * c.h * c.h);
  if (!(p.r > 0.0)) {
    p.error |= ERR_AF_RANGE;
    p.r = 1e-300;
  }
  double ns = ceil(dt * c.omega_max);
  p.n_sub = ns < 1.0 ? 1 : (ns > 1e6 ? 1000000 : (int)ns);
  *prm = p;
}

// after the projection: advance the clock
__global__ void k_end_step(Params* prm) {
  Params p = *prm;
  p.t += p.dt;
  p.dt_old = p.dt;
  p.step += 1;
  p.first = 0;
  *prm = p;
}

// ---------------------------------------------------------------- RHS (A2)
// RHS = dt [ -(alpha N^n + beta N^{n-1}) - G p^n + nu L u^n ], N in flux form.
template <class T>
__global__ void __launch_bounds__(TK* TJ)
k_rhs(Consts c, const Params* __restrict__ prm, const T* __restrict__ u,
      const T* __restrict__ v, const T* __restrict__ w, const T* __restrict__ p,
      T* __restrict__ n0, T* __restrict__ n1, T* __restrict__ n2, T* __restrict__ d0,
      T* __restrict__ d1, T* __restrict__ d2) {
  const int k = blockIdx.x * TK + threadIdx.x;
  const int j = blockIdx.y * TJ + threadIdx.y;
  if (k >= c.nz || j >= c.ny) return;
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
  const T dt = (T)prm->dt, alpha = (T)prm->alpha, beta = (T)prm->beta;
  const T nu = (T)c.nu, ih = (T)c.inv_h, ih2 = (T)(c.inv_h * c.inv_h), hf = (T)0.5;
  const size_t P = plane(c);
  auto at = [&](int i, int jj, int kk) { return ((size_t)i * ny + jj) * nz + kk; };
  const int i0 = blockIdx.z * XCHUNK;
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
        const T vxm = i == 0 ? -vc : v[id - P];
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
        const T wxm = i == 0 ? -wc : w[id - P];
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

// ---------------------------------------------------------------- outflow (A1)
// Convective condition dq/dt + U dq/dx = 0 on the outflow plane, first-order
// upwind; the increment is kept for the x line solve.
template <class T>
__global__ void k_outflow(Consts c, const Params* __restrict__ prm, T* __restrict__ u,
                          T* __restrict__ v, T* __restrict__ w, T* __restrict__ o0,
                          T* __restrict__ o1, T* __restrict__ o2) {
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = c.ny * c.nz;
  if (jk >= P) return;
  const T cc = (T)(c.u_in * prm->dt * c.inv_h);
  const size_t last = (size_t)c.nx * P + jk, prev = last - P;
  T inc = -cc * (u[last] - u[prev]);
  u[last] += inc;
  o0[jk] = inc;
  inc = -cc * (v[last] - v[prev]);
  v[last] += inc;
  o1[jk] = inc;
  inc = -cc * (w[last] - w[prev]);
  w[last] += inc;
  o2[jk] = inc;
}

// ---------------------------------------------------------------- implicit factors (A3)
// Each factor (1 - a L_d) is (r / 1)(q x_k - x_{k-1} - x_{k+1}) with
// q = 2 + 1/r = rho + 1/rho, rho = exp(-theta), theta = 2 asinh(1 / (2 sqrt r)).
// x lines (Dirichlet start for u, inflow-reflection start for v, w) use the
// closed-form LU pivots p_k; periodic y, z lines use the factorisation
// q - S - S^{-1} = (1/rho)(1 - rho S^{-1})(1 - rho S) as two first-order
// recursions with periodic starting values.
__device__ inline double af_theta(double r) { return 2.0 * asinh(0.5 / sqrt(r)); }

template <class T>
__global__ void k_af_x(Consts c, const Params* __restrict__ prm, T* __restrict__ d0,
                       T* __restrict__ d1, T* __restrict__ d2, const T* __restrict__ o0,
                       const T* __restrict__ o1, const T* __restrict__ o2) {
  extern __shared__ unsigned char smem_raw[];
  T* ip_dir = reinterpret_cast<T*>(smem_raw);   // [1 .. nx-1]
  T* ip_gh = ip_dir + (c.nx + 1);               // [1 .. nx]
  const double r = prm->r;
  const double th = af_theta(r);
  const double rho = exp(-th);
  for (int kk = 1 + threadIdx.x; kk <= c.nx; kk += blockDim.x) {
    ip_dir[kk] = (T)(rho * expm1(-2.0 * kk * th) / expm1(-(2.0 * kk + 2.0) * th));
    ip_gh[kk] = (T)(rho * expm1(-(2.0 * kk - 1.0) * th) / expm1(-(2.0 * kk + 1.0) * th));
  }
  __syncthreads();
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  const int comp = blockIdx.y;
  if (jk >= P) return;
  const T ir = (T)(1.0 / r);
  const int nx = c.nx;
  if (comp == 0) {
    T* d = d0 + jk;
    T y = 0;
    for (int i = 1; i <= nx - 1; ++i) {
      T e = d[(size_t)i * P] * ir;
      if (i == nx - 1) e += o0[jk];
      y = (e + y) * ip_dir[i];
      d[(size_t)i * P] = y;
    }
    T x = 0;
    for (int i = nx - 1; i >= 1; --i) {
      x = d[(size_t)i * P] + x * ip_dir[i];
      d[(size_t)i * P] = x;
    }
  } else {
    T* d = (comp == 1 ? d1 : d2) + jk;
    const T ob = (comp == 1 ? o1 : o2)[jk];
    T y = 0;
    for (int i = 0; i <= nx - 1; ++i) {
      T e = d[(size_t)i * P] * ir;
      if (i == nx - 1) e += ob;
      y = (e + y) * ip_gh[i + 1];
      d[(size_t)i * P] = y;
    }
    T x = 0;
    for (int i = nx - 1; i >= 0; --i) {
      x = d[(size_t)i * P] + x * ip_gh[i + 1];
      d[(size_t)i * P] = x;
    }
  }
}

// periodic line solve along a strided line of n values starting at `d`
template <class T>
__device__ inline void periodic_line(T* d, int n, size_t stride, double r) {
  const double th = af_theta(r);
  const T rho = (T)exp(-th);
  const T inv1m = (T)(-1.0 / expm1(-(double)n * th));
  const T ir = (T)(1.0 / r);
  // y = (1 - rho S^{-1})^{-1} e, periodic: y_0 = sum_m rho^m e_{-m} / (1 - rho^n)
  T acc = 0, pw = 1;
  for (int m = 0; m < n; ++m) {
    if (pw < (T)1e-30) break;
    acc += pw * d[(size_t)((n - m) % n) * stride];
    pw *= rho;
  }
  T y = acc * ir * inv1m;
  d[0] = y;
  for (int jj = 1; jj < n; ++jj) {
    y = d[(size_t)jj * stride] * ir + rho * y;
    d[(size_t)jj * stride] = y;
  }
  // z = (1 - rho S)^{-1} y, periodic: z_{n-1} = sum_m rho^m y_{n-1+m} / (1 - rho^n)
  acc = 0;
  pw = 1;
  for (int m = 0; m < n; ++m) {
    if (pw < (T)1e-30) break;
    acc += pw * d[(size_t)((n - 1 + m) % n) * stride];
    pw *= rho;
  }
  T z = acc * inv1m;
  d[(size_t)(n - 1) * stride] = rho * z;
  for (int jj = n - 2; jj >= 0; --jj) {
    z = d[(size_t)jj * stride] + rho * z;
    d[(size_t)jj * stride] = rho * z;
  }
}

// y lines: one thread per (i, k), walking y with stride nz (coalesced in k)
template <class T>
__global__ void k_af_y(Consts c, const Params* __restrict__ prm, T* __restrict__ d0,
                       T* __restrict__ d1, T* __restrict__ d2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  const int comp = blockIdx.z;
  if (k >= c.nz) return;
  if (comp == 0 ? (i < 1 || i > c.nx - 1) : (i > c.nx - 1)) return;
  T* d = (comp == 0 ? d0 : (comp == 1 ? d1 : d2)) + (size_t)i * plane(c) + k;
  periodic_line(d, c.ny, (size_t)c.nz, prm->r);
}

// z lines are contiguous: a block stages ZL lines in shared memory, one
// thread per line solves, then u* = u^n + du is written back.
constexpr int ZL = 32;
template <class T>
__global__ void __launch_bounds__(128)
k_af_z(Consts c, const Params* __restrict__ prm, T* __restrict__ d0, T* __restrict__ d1,
       T* __restrict__ d2, T* __restrict__ u, T* __restrict__ v, T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int nz = c.nz, ny = c.ny;
  const int ld = nz + 1;
  const int comp = blockIdx.y;
  const int first = comp == 0 ? ny : 0;               // u: planes 1..nx-1
  const int last = c.nx * ny;                          // exclusive
  const int L0 = first + blockIdx.x * ZL;
  if (L0 >= last) return;
  const int nl = min(ZL, last - L0);
  T* d = comp == 0 ? d0 : (comp == 1 ? d1 : d2);
  T* q = comp == 0 ? u : (comp == 1 ? v : w);
  const size_t base = (size_t)L0 * nz;
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    const int l = e / nz, kk = e - l * nz;
    s[l * ld + kk] = d[base + e];
  }
  __syncthreads();
  if (threadIdx.x < nl) periodic_line(s + threadIdx.x * ld, nz, 1, prm->r);
  __syncthreads();
  for (int e = threadIdx.x; e < nl * nz; e += blockDim.x) {
    const int l = e / nz, kk = e - l * nz;
    q[base + e] += s[l * ld + kk];
  }
}

// ---------------------------------------------------------------- mass fix + divergence (A7)
// Q_in, Q_out over the inflow/outflow faces (FP64, fixed summation order);
// the shift (Q_in - Q_out) / (Ly Lz) goes onto the outflow face.
template <class T>
__global__ void k_mass(Consts c, Params* prm, const T* __restrict__ u) {
  __shared__ double scratch[32];
  const int P = c.ny * c.nz;
  double qi = 0.0, qo = 0.0;
  const T* u0 = u;
  const T* un = u + (size_t)c.nx * P;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    qi += (double)u0[e];
    qo += (double)un[e];
  }
  qi = block_sum(qi, scratch);
  __syncthreads();
  qo = block_sum(qo, scratch);
  if (threadIdx.x == 0) {
    const double h2 = c.h * c.h;
    prm->q_in = qi * h2;
    prm->q_out = qo * h2;
    prm->mass_shift = (qi - qo) * h2 / (c.ly * c.lz);
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
  const T shift = initial ? (T)0 : (T)prm->mass_shift;
  const T sc = (T)(c.inv_h / (initial ? 1.0 : prm->dt));
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
          T* __restrict__ vb, T* __restrict__ wb, const T* __restrict__ phi, T* __restrict__ p,
          double* __restrict__ partial, int initial) {
  const int k = blockIdx.x * TK + threadIdx.x;
  const int j = blockIdx.y * TJ + threadIdx.y;
  const bool act = (k < c.nz && j < c.ny);
  const int ny = c.ny, nz = c.nz, nx = c.nx;
  const size_t P = plane(c);
  double smax = 0.0;
  if (act) {
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
    const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
    const T dt = initial ? (T)1 : (T)prm->dt;
    const T gdt = dt * (T)c.inv_h;
    const T hnu = initial ? (T)0 : (T)(0.5 * c.nu * prm->dt * c.inv_h * c.inv_h);
    auto at = [&](int i, int jj, int kk) { return ((size_t)i * ny + jj) * nz + kk; };
    auto unew = [&](int i) -> T {  // new u on face i at (j, k)
      const size_t id = at(i, j, k);
      if (i >= 1 && i <= nx - 1) return ua[id] - gdt * (phi[id] - phi[id - P]);
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
      const T ph = phi[id];
      const T vn = va[id] - gdt * (ph - phi[at(i, jm, k)]);
      const T wn = wa[id] - gdt * (ph - phi[at(i, j, km)]);
      vb[id] = vn;
      wb[id] = wn;
      if (!initial) {
        const T pxm = i == 0 ? ph : phi[id - P];
        const T pxp = i == nx - 1 ? ph : phi[id + P];
        const T lap = pxm + pxp + phi[at(i, jm, k)] + phi[at(i, jp, k)] + phi[at(i, j, km)] +
                      phi[at(i, j, kp)] - (T)6 * ph;
        p[id] += ph - hnu * lap;
      }
      const T un1 = unew(i + 1);
      const T vn1 = va[at(i, jp, k)] - gdt * (phi[at(i, jp, k)] - ph);
      const T wn1 = wa[at(i, j, kp)] - gdt * (phi[at(i, j, kp)] - ph);
      double sp = fabs(0.5 * ((double)un + (double)un1)) + fabs(0.5 * ((double)vn + (double)vn1)) +
                  fabs(0.5 * ((double)wn + (double)wn1));
      if (!isfinite(sp)) sp = INFINITY;
      smax = fmax(smax, sp);
    }
  }
  // flatten the 2-D block for the reduction
  const int tid = threadIdx.y * TK + threadIdx.x;
  double v = warp_max(smax);
  __shared__ double wmax[TK * TJ / 32];
  if ((tid & 31) == 0) wmax[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int q = 0; q < TK * TJ / 32; ++q) m = fmax(m, wmax[q]);
    partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = m;
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

template <class T>
void launch_begin_step(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  k_begin_step<<<1, 1024, 0, s>>>(c, f.prm, f.partial, f.n_partial);
}

template <class T>
void launch_rhs(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  k_rhs<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur],
                                                        f.p, f.n[0], f.n[1], f.n[2], f.d[0],
                                                        f.d[1], f.d[2]);
}

template <class T>
void launch_outflow(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  const int P = c.ny * c.nz;
  k_outflow<T><<<(P + 255) / 256, 256, 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.dout[0],
                                                f.dout[1], f.dout[2]);
}

template <class T>
void launch_af_x(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  const int P = c.ny * c.nz;
  const size_t shx = 2 * (size_t)(c.nx + 1) * sizeof(T);
  k_af_x<T><<<dim3((P + 127) / 128, 3), 128, shx, s>>>(c, f.prm, f.d[0], f.d[1], f.d[2],
                                                        f.dout[0], f.dout[1], f.dout[2]);
  (void)cur;
}

template <class T>
void launch_af_y(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  k_af_y<T><<<dim3((c.nz + 63) / 64, c.nx, 3), 64, 0, s>>>(c, f.prm, f.d[0], f.d[1], f.d[2]);
  (void)cur;
}

template <class T>
void launch_af_z(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  const size_t shz = (size_t)ZL * (c.nz + 1) * sizeof(T);
  k_af_z<T><<<dim3((c.nx * c.ny + ZL - 1) / ZL, 3), 128, shz, s>>>(
      c, f.prm, f.d[0], f.d[1], f.d[2], f.u[cur], f.v[cur], f.w[cur]);
}

template <class T>
void launch_af(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  launch_af_x(c, f, cur, s);
  launch_af_y(c, f, cur, s);
  launch_af_z(c, f, cur, s);
}

template <class T>
void launch_mass(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s) {
  k_mass<T><<<1, 1024, 0, s>>>(c, f.prm, f.u[cur]);
}

template <class T>
void launch_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  k_div<T><<<grid3(c, c.nx), dim3(TK, TJ), 0, s>>>(c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.phi,
                                                    initial ? 1 : 0);
}

template <class T>
void launch_mass_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  if (!initial) launch_mass(c, f, cur, s);
  launch_div(c, f, cur, initial, s);
}

template <class T>
void launch_project_only(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  k_project<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(
      c, f.prm, f.u[cur], f.v[cur], f.w[cur], f.u[cur ^ 1], f.v[cur ^ 1], f.w[cur ^ 1], f.phi, f.p,
      f.partial, initial ? 1 : 0);
}

template <class T>
void launch_project(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s) {
  launch_project_only(c, f, cur, initial, s);
  if (!initial) k_end_step<<<1, 1, 0, s>>>(f.prm);
}

template <class T>
void launch_stats(const Consts& c, const Fields<T>& f, int cur, double* out, cudaStream_t s) {
  k_stats<T><<<grid3(c, c.nx + 1), dim3(TK, TJ), 0, s>>>(c, f.u[cur], f.v[cur], f.w[cur], out);
}

void fluid_set_attributes() {
  cudaFuncSetAttribute(k_af_z<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_z<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_x<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_af_x<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int partial_count(const Consts& c) {
  const dim3 g = grid3(c, c.nx + 1);
  return (int)(g.x * g.y * g.z);
}

#define INST(T)                                                                                \
  template void launch_begin_step<T>(const Consts&, const Fields<T>&, cudaStream_t);           \
  template void launch_rhs<T>(const Consts&, const Fields<T>&, int, cudaStream_t);             \
  template void launch_outflow<T>(const Consts&, const Fields<T>&, int, cudaStream_t);         \
  template void launch_af<T>(const Consts&, const Fields<T>&, int, cudaStream_t);              \
  template void launch_af_x<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_af_y<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_af_z<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_mass<T>(const Consts&, const Fields<T>&, int, cudaStream_t);            \
  template void launch_div<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t);       \
  template void launch_project_only<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t); \
  template void launch_mass_div<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t);  \
  template void launch_project<T>(const Consts&, const Fields<T>&, int, bool, cudaStream_t);   \
  template void launch_stats<T>(const Consts&, const Fields<T>&, int, double*, cudaStream_t);
INST(double)
INST(float)

}  // namespace ibm
