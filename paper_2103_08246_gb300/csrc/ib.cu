// Immersed-boundary direct forcing (Sec. II.B): interpolation of the
// provisional velocity at every marker (a gather over the 3 x 3 x 3 nodes of
// each staggered lattice in the support of the three-point kernel of Roma,
// Peskin and Berger), the direct-forcing amplitude
//   coef_l = dV_l / h^3 (U_l - U*_l)   (= dt F_l dV_l / h^3),
// the fluid force on each flag vertex -F_l dV_l, and spreading of coef_l
// with the same weights (atomic scatter). Alternatively the bars are forced
// on the Eulerian nodes (k_bar_mask) and only the flag carries markers.
//
// Markers 0 .. nf-1 are the flag vertices (target velocity V_l, position X_l
// from the structure), the rest the bar-grid markers (target 0). Nodes
// outside the unknowns along x are skipped (u faces 0 and nx, the v/w ghost
// plane); y and z wrap periodically. Non-finite positions are skipped, so a
// diverged flag cannot produce an out-of-range access.
#include <cmath>

#include "solver.h"

namespace ibm {

template <class T>
__device__ inline T roma_phi(T r) {
  const T a = fabs(r);
  if (a <= (T)0.5) return ((T)1 + sqrt((T)1 - (T)3 * a * a)) / (T)3;
  if (a < (T)1.5) {
    const T b = (T)1 - a;
    return ((T)5 - (T)3 * a - sqrt(fmax((T)0, (T)1 - (T)3 * b * b))) / (T)6;
  }
  return (T)0;
}

// 64-bit fixed point of the deterministic scatter: value * 2^40, two's
// complement in an unsigned word (integer addition wraps identically)
constexpr double FIX_SCALE = 1099511627776.0;   // 2^40
__device__ inline unsigned long long to_fixed(double x) {
  return (unsigned long long)__double2ll_rn(x * FIX_SCALE);
}
__device__ inline unsigned long long to_fixed(float x) {
  return (unsigned long long)__float2ll_rn(x * (float)FIX_SCALE);
}
template <class T>
__device__ inline T from_fixed(unsigned long long s) {
  return (T)((double)(long long)s * (1.0 / FIX_SCALE));
}

struct Stencil {
  int i0, j[3], k[3];
  bool vi[3];
};

// Per marker and direction: base node index and fractional offset of the
// two staggered lattices (node offset 0 and 1/2), computed once in FP64;
// weights phi(t - 1/2 - f), t = 0, 1, 2, then follow in the field precision.
template <class T>
struct Frac {
  int i0[2];
  T f[2];
};
template <class T>
__device__ inline Frac<T> frac_of(double s) {   // s = X / h
  Frac<T> r;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const double a = s - 0.5 * o - 0.5;
    const double fl = floor(a);
    r.i0[o] = (int)fl;
    r.f[o] = (T)(a - fl);
  }
  return r;
}

// 3-node stencil per direction of component `comp`
template <class T>
__device__ inline void stencil(const Consts& c, int comp, const Frac<T>& fx, const Frac<T>& fy,
                               const Frac<T>& fz, Stencil& st, T wx[3], T wy[3], T wz[3]) {
  const int ox = comp == 0 ? 0 : 1, oy = comp == 1 ? 0 : 1, oz = comp == 2 ? 0 : 1;
  const int ix = fx.i0[ox], iy = fy.i0[oy], iz = fz.i0[oz];
  const int lo = comp == 0 ? 1 : 0, hi = c.nx - 1;
  st.i0 = ix;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const T tt = (T)t - (T)0.5;
    wx[t] = roma_phi<T>(tt - fx.f[ox]);
    wy[t] = roma_phi<T>(tt - fy.f[oy]);
    wz[t] = roma_phi<T>(tt - fz.f[oz]);
    st.vi[t] = (ix + t >= lo) && (ix + t <= hi);
    int jj = (iy + t) % c.ny;
    if (jj < 0) jj += c.ny;
    int kk = (iz + t) % c.nz;
    if (kk < 0) kk += c.nz;
    st.j[t] = jj;
    st.k[t] = kk;
  }
}

__device__ inline bool marker(const Markers& m, const Flag& fl, int l, double& X, double& Y,
                              double& Z, double U[3], double& dv) {
  if (l < m.nf) {
    X = fl.X[3 * l];
    Y = fl.X[3 * l + 1];
    Z = fl.X[3 * l + 2];
    U[0] = fl.V[3 * l];
    U[1] = fl.V[3 * l + 1];
    U[2] = fl.V[3 * l + 2];
    dv = fl.dv[l];
  } else {
    const int b = l - m.nf;
    X = m.Xb[3 * b];
    Y = m.Xb[3 * b + 1];
    Z = m.Xb[3 * b + 2];
    U[0] = U[1] = U[2] = 0.0;
    dv = m.bar_dv;
  }
  // finite and inside a generous box: otherwise skip
  return isfinite(X) && isfinite(Y) && isfinite(Z) && fabs(X) < 1e6 && fabs(Y) < 1e6 &&
         fabs(Z) < 1e6;
}

template <class T>
__global__ void k_ib_interp(Consts c, Params* prm, Markers m, Flag fl, const T* __restrict__ u,
                            const T* __restrict__ v, const T* __restrict__ w) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l == 0 && m.nf > 0) {   // hand this step's dt to the pending structural update
    prm->flag_dt = prm->dt;
    prm->flag_nsub = prm->n_sub;
    prm->flag_pending = 1;
  }
  double slip = 0.0;
  if (l < m.nm) {
    double X, Y, Z, U[3], dv;
    const bool ok = marker(m, fl, l, X, Y, Z, U, dv);
    double us[3] = {0.0, 0.0, 0.0};
    if (ok) {
      const Frac<T> fx = frac_of<T>(X * c.inv_h), fy = frac_of<T>(Y * c.inv_h),
                    fz = frac_of<T>(Z * c.inv_h);
      for (int comp = 0; comp < 3; ++comp) {
        const T* q = comp == 0 ? u : (comp == 1 ? v : w);
        Stencil st;
        T wx[3], wy[3], wz[3];
        stencil<T>(c, comp, fx, fy, fz, st, wx, wy, wz);
        T acc = 0;
        for (int a = 0; a < 3; ++a) {
          if (!st.vi[a]) continue;
          const size_t pi = (size_t)(st.i0 + a) * c.ny;
          for (int b = 0; b < 3; ++b) {
            const size_t pj = (pi + st.j[b]) * c.nz;
            const T wab = wx[a] * wy[b];
            for (int e = 0; e < 3; ++e) acc += wab * wz[e] * q[pj + st.k[e]];
          }
        }
        us[comp] = (double)acc;
      }
    }
    const double vol = dv * c.inv_h * c.inv_h * c.inv_h;
    const double dt = prm->dt;
    for (int comp = 0; comp < 3; ++comp) {
      const double du = ok ? (U[comp] - us[comp]) : 0.0;
      m.coef[3 * l + comp] = vol * du;
      if (l < m.nf) fl.Ff[3 * l + comp] = -du / dt * dv;
      slip = fmax(slip, fabs(du));
    }
  }
  slip = warp_max(slip);
  if ((threadIdx.x & 31) == 0 && slip > 0.0) atomic_max_nonneg(&prm->slip_max, slip);
}

template <class T>
__global__ void k_ib_spread(Consts c, Markers m, Flag fl, T* __restrict__ u, T* __restrict__ v,
                            T* __restrict__ w) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m.nm) return;
  double X, Y, Z, U[3], dv;
  if (!marker(m, fl, l, X, Y, Z, U, dv)) return;
  const Frac<T> fx = frac_of<T>(X * c.inv_h), fy = frac_of<T>(Y * c.inv_h),
                fz = frac_of<T>(Z * c.inv_h);
  for (int comp = 0; comp < 3; ++comp) {
    const T cf = (T)m.coef[3 * l + comp];
    if (cf == (T)0) continue;
    T* q = comp == 0 ? u : (comp == 1 ? v : w);
    Stencil st;
    T wx[3], wy[3], wz[3];
    stencil<T>(c, comp, fx, fy, fz, st, wx, wy, wz);
    for (int a = 0; a < 3; ++a) {
      if (!st.vi[a] || wx[a] == (T)0) continue;
      const size_t pi = (size_t)(st.i0 + a) * c.ny;
      for (int b = 0; b < 3; ++b) {
        const T wab = wx[a] * wy[b] * cf;
        if (wab == (T)0) continue;
        const size_t pj = (pi + st.j[b]) * c.nz;
        for (int e = 0; e < 3; ++e) {
          const T val = wab * wz[e];
          if (val == (T)0) continue;
          if (m.acc)
            atomicAdd(&m.acc[comp * m.nfield + pj + st.k[e]], to_fixed(val));
          else
            atomicAdd(&q[pj + st.k[e]], val);
        }
      }
    }
  }
}

// Deterministic mode, second pass: every node a marker touched takes its
// fixed-point sum out of the accumulator (exchange with zero); the first
// visitor adds it to the field, later visitors find zero. One nonzero
// addition per node: the result does not depend on thread order.
template <class T>
__global__ void k_ib_flush(Consts c, Markers m, Flag fl, T* __restrict__ u, T* __restrict__ v,
                           T* __restrict__ w) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m.nm) return;
  double X, Y, Z, U[3], dv;
  if (!marker(m, fl, l, X, Y, Z, U, dv)) return;
  const Frac<T> fx = frac_of<T>(X * c.inv_h), fy = frac_of<T>(Y * c.inv_h),
                fz = frac_of<T>(Z * c.inv_h);
  for (int comp = 0; comp < 3; ++comp) {
    T* q = comp == 0 ? u : (comp == 1 ? v : w);
    Stencil st;
    T wx[3], wy[3], wz[3];
    stencil<T>(c, comp, fx, fy, fz, st, wx, wy, wz);
    for (int a = 0; a < 3; ++a) {
      if (!st.vi[a]) continue;
      const size_t pi = (size_t)(st.i0 + a) * c.ny;
      for (int b = 0; b < 3; ++b) {
        const size_t pj = (pi + st.j[b]) * c.nz;
        for (int e = 0; e < 3; ++e) {
          const unsigned long long sum = atomicExch(&m.acc[comp * m.nfield + pj + st.k[e]], 0ull);
          if (sum != 0ull) atomicAdd(&q[pj + st.k[e]], from_fixed<T>(sum));
        }
      }
    }
  }
}

// Eulerian direct forcing of the bar grid (Sec. II.B, the fixed grid forced
// on Eulerian nodes): u** = (1 - alpha) u* at every velocity node whose cell
// the bars cut, alpha the cell's solid fraction (zero velocity inside)
template <class T>
__global__ void k_bar_mask(Markers m, T* __restrict__ u, T* __restrict__ v, T* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n0 = m.nbm[0], n1 = n0 + m.nbm[1], n2 = n1 + m.nbm[2];
  if (i >= n2) return;
  T* q = i < n0 ? u : (i < n1 ? v : w);
  q[m.bm_idx[i]] *= (T)(1.0 - m.bm_alpha[i]);
}

template <class T>
void launch_ib(const Consts& c, const Fields<T>& f, const Markers& m, const Flag& fl, int cur,
               cudaStream_t s) {
  const int nbm = m.nbm[0] + m.nbm[1] + m.nbm[2];
  if (nbm) k_bar_mask<T><<<(nbm + 255) / 256, 256, 0, s>>>(m, f.u[cur], f.v[cur], f.w[cur]);
  if (m.nm == 0) return;
  const int nb = (m.nm + 127) / 128;
  k_ib_interp<T><<<nb, 128, 0, s>>>(c, f.prm, m, fl, f.u[cur], f.v[cur], f.w[cur]);
  k_ib_spread<T><<<nb, 128, 0, s>>>(c, m, fl, f.u[cur], f.v[cur], f.w[cur]);
  if (m.acc) k_ib_flush<T><<<nb, 128, 0, s>>>(c, m, fl, f.u[cur], f.v[cur], f.w[cur]);
}

template void launch_ib<double>(const Consts&, const Fields<double>&, const Markers&, const Flag&,
                                int, cudaStream_t);
template void launch_ib<float>(const Consts&, const Fields<float>&, const Markers&, const Flag&,
                               int, cudaStream_t);

}  // namespace ibm
