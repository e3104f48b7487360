// Immersed-boundary direct forcing (Sec. II.B): interpolation of the
// provisional velocity at every marker (a gather over the 3 x 3 x 3 nodes of
// each staggered lattice in the support of the three-point kernel of Roma,
// Peskin and Berger), the direct-forcing amplitude
//   coef_l = dV_l / h^3 (U_l - U*_l)   (= dt F_l dV_l / h^3),
// the fluid force on each flag vertex -F_l dV_l, and spreading of coef_l
// with the same weights (atomic scatter). Alternatively the bars are forced
// on the Eulerian nodes (k_bar_mask) and only the flag carries markers.
//
// The bar-grid markers never move: they are binned once into tiles of
// TX x TY x TZ cells (sorted by tile, host side). Per tile, one block stages
// the velocity box the tile's kernels can reach ((T + 3)^3 nodes per
// component) in shared memory and interpolates from it; the spreading block
// accumulates the tile's contributions in a shared-memory box and adds each
// nonzero node to the field once (one coalesced atomic per node and tile
// instead of 27 scattered ones per marker and component). The flag's moving
// markers take one thread each in extra blocks of the same launches.
//
// Markers 0 .. nf-1 are the flag vertices (target velocity V_l, position X_l
// from the structure), the rest the bar-grid markers (target 0). Nodes
// outside the unknowns along x are skipped (u faces 0 and nx, the v/w ghost
// plane); y and z wrap periodically. Non-finite positions are skipped, so a
// diverged flag cannot produce an out-of-range access.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "async_copy.cuh"
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
    X = fl.X[3 * l] - m.x_shift;
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

// ---------------------------------------------------------------- tiled bars
// Box of a tile: cells [o, o + T) in each direction reach nodes [o - 1, o + T + 1]
// (the three-node stencils of both staggered lattices), B = T + 3 nodes.
struct TileBox {
  int ox, oy, oz;   // grid coordinates of box node (0, 0, 0) (y, z unwrapped)
  int bx, by, bz, n;
  int b0, b1;       // bar markers of the tile (bar indices)
};
__device__ inline TileBox tile_box(const Markers& m, int t) {
  const int* ti = m.tile + 5 * t;
  TileBox b;
  b.ox = ti[0] - 1;
  b.oy = ti[1] - 1;
  b.oz = ti[2] - 1;
  b.bx = m.tx + 3;
  b.by = m.ty + 3;
  b.bz = m.tz + 3;
  b.n = b.bx * b.by * b.bz;
  b.b0 = ti[3];
  b.b1 = ti[4];
  return b;
}
__device__ inline int pos_mod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// interpolation, amplitude and flag force of one marker from global memory
template <class T>
__device__ inline double interp_marker(const Consts& c, const Params* prm, const Markers& m,
                                       const Flag& fl, int l, const T* __restrict__ u,
                                       const T* __restrict__ v, const T* __restrict__ w) {
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
  double slip = 0.0;
  for (int comp = 0; comp < 3; ++comp) {
    const double du = ok ? (U[comp] - us[comp]) : 0.0;
    m.coef[3 * l + comp] = vol * du;
    if (l < m.nf) fl.Ff[3 * l + comp] = -du / dt * dv;
    slip = fmax(slip, fabs(du));
  }
  return slip;
}

// Per bar marker, once at set-up (the markers never move): the kernel
// weights phi(t - 1/2 - f) of both staggered lattices (offset 0 and 1/2) in
// each direction, 18 values in the field precision (slot (3 d + t) for
// offset 0, 9 + (3 d + t) for offset 1/2, marker-fastest), and the stencils'
// first box indices, 5 bits per (offset, direction), packed in one int.
// Computed exactly as the per-marker kernels compute them.
template <class T>
__global__ void __launch_bounds__(256)
k_ib_bar_setup(Consts c, Params* prm, Markers m, T* __restrict__ bw, int* __restrict__ bo) {
  const TileBox bx = tile_box(m, blockIdx.x);
  const size_t nb = (size_t)m.nb;
  for (int b = bx.b0 + threadIdx.x; b < bx.b1; b += blockDim.x) {
    const double Xs[3] = {m.Xb[3 * b] * c.inv_h, m.Xb[3 * b + 1] * c.inv_h, m.Xb[3 * b + 2] * c.inv_h};
    const int org[3] = {bx.ox, bx.oy, bx.oz}, lim[3] = {bx.bx - 3, bx.by - 3, bx.bz - 3};
    const int per[3] = {0, c.ny, c.nz};
    int packed = 0;
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
      const Frac<T> f = frac_of<T>(Xs[d]);
      for (int o = 0; o < 2; ++o) {
        int r = f.i0[o] - org[d];
        if (d > 0) r = pos_mod(r, per[d]);
        ok = ok && r >= 0 && r <= lim[d];
        packed |= (r & 31) << (5 * (3 * o + d));
        for (int t = 0; t < 3; ++t)
          bw[(size_t)(9 * o + 3 * d + t) * nb + b] = roma_phi<T>((T)t - (T)0.5 - f.f[o]);
      }
    }
    bo[b] = packed;
    if (!ok) atomicOr(&prm->error, ERR_IB_BIN);
  }
}

// box offset and weights of a bar marker's stencil on component comp (the
// lattice offset is 0 along comp, 1/2 across)
template <class T>
__device__ inline int bar_stencil(const Markers& m, const TileBox& bx, const T* __restrict__ bw, int packed,
                                  int b, int comp, T wx[3], T wy[3], T wz[3]) {
  const size_t nb = (size_t)m.nb;
  const int ox = comp == 0 ? 0 : 1, oy = comp == 1 ? 0 : 1, oz = comp == 2 ? 0 : 1;
  const int rx = (packed >> (5 * (3 * ox))) & 31, ry = (packed >> (5 * (3 * oy + 1))) & 31,
            rz = (packed >> (5 * (3 * oz + 2))) & 31;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    wx[t] = bw[(size_t)(9 * ox + t) * nb + b];
    wy[t] = bw[(size_t)(9 * oy + 3 + t) * nb + b];
    wz[t] = bw[(size_t)(9 * oz + 6 + t) * nb + b];
  }
  return comp * bx.n + (rx * bx.by + ry) * bx.bz + rz;
}

// rows (component, x, y) of the tile box, one warp per row, lanes along z;
// f(box index, field index or -1, component). The row coordinates advance
// by the warp count with carries (no divisions); a tile starts inside the
// periodic range and spans at most its own length beyond it, so one
// conditional wrap per coordinate suffices.
template <class F>
__device__ inline void for_box_rows(const Consts& c, const TileBox& bx, F f) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int rows = 3 * bx.bx * bx.by;
  int row = threadIdx.x >> 5;
  int comp = 0, a = 0, bb = row;
  while (bb >= bx.by) {
    bb -= bx.by;
    if (++a == bx.bx) a = 0, ++comp;
  }
  int k = bx.oz + lane;
  if (k < 0) k += c.nz;
  if (k >= c.nz) k -= c.nz;
  const bool lane_on = lane < bx.bz;
  for (; row < rows; row += nw) {
    const int i = bx.ox + a;
    int j = bx.oy + bb;
    if (j < 0) j += c.ny;
    if (j >= c.ny) j -= c.ny;
    const bool xin = i >= (comp == 0 ? 1 : 0) && i <= c.nx - 1;
    if (lane_on) f(row * bx.bz + lane, xin ? (long long)idx3(c, i, j, k) : -1ll, comp);
    bb += nw;
    while (bb >= bx.by) {
      bb -= bx.by;
      if (++a == bx.bx) a = 0, ++comp;
    }
  }
}

// blocks 0 .. n_tiles-1: one bar tile each (velocity box staged in shared
// memory); further blocks: one flag marker per thread
constexpr int IB_THREADS = 512;
template <class T>
__global__ void __launch_bounds__(IB_THREADS)
k_ib_interp_tiles(Consts c, Params* prm, Markers m, Flag fl, const T* __restrict__ bw,
                  const int* __restrict__ bo, const T* __restrict__ u, const T* __restrict__ v,
                  const T* __restrict__ w) {
  extern __shared__ __align__(16) unsigned char ib_smem[];
  T* box = reinterpret_cast<T*>(ib_smem);
  if (blockIdx.x == 0 && threadIdx.x == 0 && m.nf > 0) {   // hand this step's dt to the structure
    prm->flag_dt = prm->dt;
    prm->flag_nsub = prm->n_sub;
    prm->flag_pending = 1;
  }
  double slip = 0.0;
  if ((int)blockIdx.x >= m.n_tiles) {
    const int l = ((int)blockIdx.x - m.n_tiles) * blockDim.x + threadIdx.x;
    if (l < m.nf) slip = interp_marker<T>(c, prm, m, fl, l, u, v, w);
  } else {
    const TileBox bx = tile_box(m, blockIdx.x);
    // every copy in flight at once (cp.async), one wait
    const uint32_t sb = smem_u32(box);
    for_box_rows(c, bx, [&](int q, long long g, int comp) {
      const T* src = comp == 0 ? u : (comp == 1 ? v : w);
      if (g >= 0)
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sb + (uint32_t)(q * sizeof(T))),
                     "l"(src + g), "n"(sizeof(T))
                     : "memory");
      else
        box[q] = (T)0;
    });
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const double vol = m.bar_dv * c.inv_h * c.inv_h * c.inv_h;
    for (int b = bx.b0 + threadIdx.x; b < bx.b1; b += blockDim.x) {
      const int packed = bo[b];
      const int l = m.nf + b;
      for (int comp = 0; comp < 3; ++comp) {
        T wx[3], wy[3], wz[3];
        const T* bq = box + bar_stencil<T>(m, bx, bw, packed, b, comp, wx, wy, wz);
        T acc = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int e2 = 0; e2 < 3; ++e2) {
            const T wab = wx[a] * wy[e2];
            const T* row = bq + (a * bx.by + e2) * bx.bz;
#pragma unroll
            for (int e = 0; e < 3; ++e) acc += wab * wz[e] * row[e];
          }
        const double du = -(double)acc;
        m.coef[3 * l + comp] = vol * du;
        slip = fmax(slip, fabs(du));
      }
    }
  }
  slip = warp_max(slip);
  if ((threadIdx.x & 31) == 0 && slip > 0.0) atomic_max_nonneg(&prm->slip_max, slip);
}

// spreading: per bar tile, contributions summed in a shared-memory box, then
// every nonzero node added to the field with one atomic; flag markers one
// per thread with global atomics (all additions commute)
template <class T>
__global__ void __launch_bounds__(IB_THREADS)
k_ib_spread_tiles(Consts c, Markers m, Flag fl, const T* __restrict__ bw, const int* __restrict__ bo,
                  T* __restrict__ u, T* __restrict__ v, T* __restrict__ w) {
  extern __shared__ __align__(16) unsigned char ib_smem[];
  T* box = reinterpret_cast<T*>(ib_smem);
  if ((int)blockIdx.x >= m.n_tiles) {
    const int l = ((int)blockIdx.x - m.n_tiles) * blockDim.x + threadIdx.x;
    if (l >= m.nf) return;
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
        if (!st.vi[a]) continue;
        const size_t pi = (size_t)(st.i0 + a) * c.ny;
        for (int b = 0; b < 3; ++b) {
          const T wab = wx[a] * wy[b] * cf;
          const size_t pj = (pi + st.j[b]) * c.nz;
          for (int e = 0; e < 3; ++e) atomicAdd(&q[pj + st.k[e]], wab * wz[e]);
        }
      }
    }
    return;
  }
  const TileBox bx = tile_box(m, blockIdx.x);
  for (int q = threadIdx.x; q < 3 * bx.n; q += blockDim.x) box[q] = (T)0;
  __syncthreads();
  for (int b = bx.b0 + threadIdx.x; b < bx.b1; b += blockDim.x) {
    const int packed = bo[b];
    const int l = m.nf + b;
    for (int comp = 0; comp < 3; ++comp) {
      T wx[3], wy[3], wz[3];
      T* bq = box + bar_stencil<T>(m, bx, bw, packed, b, comp, wx, wy, wz);
      const T cf = (T)m.coef[3 * l + comp];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e2 = 0; e2 < 3; ++e2) {
          const T wab = wx[a] * wy[e2] * cf;
          T* row = bq + (a * bx.by + e2) * bx.bz;
#pragma unroll
          for (int e = 0; e < 3; ++e) atomicAdd(&row[e], wab * wz[e]);
        }
    }
  }
  __syncthreads();
  for_box_rows(c, bx, [&](int q, long long g, int comp) {
    const T val = box[q];
    if (val == (T)0 || g < 0) return;
    T* dst = comp == 0 ? u : (comp == 1 ? v : w);
    atomicAdd(&dst[g], val);
  });
}

template <class T>
void launch_ib_setup(const Consts& c, const Fields<T>& f, const Markers& m, cudaStream_t s) {
  if (!m.n_tiles) return;
  k_ib_bar_setup<T><<<m.n_tiles, 256, 0, s>>>(c, f.prm, m, reinterpret_cast<T*>(m.bar_w), m.bar_o);
}
template void launch_ib_setup<double>(const Consts&, const Fields<double>&, const Markers&, cudaStream_t);
template void launch_ib_setup<float>(const Consts&, const Fields<float>&, const Markers&, cudaStream_t);

// Host: tiles of 8 x 16 x 16 cells (fewer across a short transverse side),
// starting at the lowest x cell of the bars; y, z tiles from cell 0 with
// periodic cells. A marker's cell is floor(X / h) as the kernels compute it
// (the same FP64 product), so a marker's stencils stay inside its tile's box.
void ib_bin_bars(const Consts& c, std::vector<double>& Xb, std::vector<int>& tiles, Markers& m) {
  tiles.clear();
  m.n_tiles = 0;
  const size_t nb = Xb.size() / 3;
  if (!nb) return;
  m.tx = 8;
  m.ty = c.ny < 16 ? c.ny : 16;
  m.tz = c.nz < 16 ? c.nz : 16;
  auto cell = [&](double x, int n, bool periodic) {
    long long q = (long long)std::floor(x * c.inv_h);
    if (periodic) q = ((q % n) + n) % n;
    return (int)q;
  };
  int x0 = INT32_MAX, x1 = INT32_MIN;
  for (size_t b = 0; b < nb; ++b) {
    const int cx = cell(Xb[3 * b], c.nx, false);
    x0 = std::min(x0, cx);
    x1 = std::max(x1, cx);
  }
  const int ntx = (x1 - x0) / m.tx + 1;
  const int nty = (c.ny + m.ty - 1) / m.ty, ntz = (c.nz + m.tz - 1) / m.tz;
  const size_t ntile = (size_t)ntx * nty * ntz;
  std::vector<int> key(nb), count(ntile + 1, 0);
  for (size_t b = 0; b < nb; ++b) {
    const int tx = (cell(Xb[3 * b], c.nx, false) - x0) / m.tx;
    const int ty = cell(Xb[3 * b + 1], c.ny, true) / m.ty;
    const int tz = cell(Xb[3 * b + 2], c.nz, true) / m.tz;
    key[b] = (tx * nty + ty) * ntz + tz;
    ++count[key[b] + 1];
  }
  for (size_t t = 0; t < ntile; ++t) count[t + 1] += count[t];
  std::vector<double> sorted(Xb.size());
  std::vector<int> pos(count.begin(), count.end() - 1);
  for (size_t b = 0; b < nb; ++b) {
    const int d = pos[key[b]]++;
    for (int q = 0; q < 3; ++q) sorted[3 * (size_t)d + q] = Xb[3 * b + q];
  }
  Xb.swap(sorted);
  for (size_t t = 0; t < ntile; ++t) {
    if (count[t + 1] == count[t]) continue;
    const int tz = (int)(t % ntz), ty = (int)((t / ntz) % nty), tx = (int)(t / ((size_t)ntz * nty));
    tiles.insert(tiles.end(), {x0 + tx * m.tx, ty * m.ty, tz * m.tz, count[t], count[t + 1]});
  }
  m.n_tiles = (int)(tiles.size() / 5);
}

size_t ib_tile_smem(const Markers& m, size_t elem) {
  return 3 * (size_t)(m.tx + 3) * (m.ty + 3) * (m.tz + 3) * elem;
}

void ib_set_attributes() {
  // the FP64 box of an 8 x 16 x 16 tile is 95 KB
  cudaFuncSetAttribute(k_ib_interp_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_ib_spread_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_ib_interp_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(k_ib_spread_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
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
  if (m.acc) {   // deterministic: fixed-point scatter per marker, then one addition per node
    const int nb = (m.nm + 127) / 128;
    k_ib_interp<T><<<nb, 128, 0, s>>>(c, f.prm, m, fl, f.u[cur], f.v[cur], f.w[cur]);
    k_ib_spread<T><<<nb, 128, 0, s>>>(c, m, fl, f.u[cur], f.v[cur], f.w[cur]);
    k_ib_flush<T><<<nb, 128, 0, s>>>(c, m, fl, f.u[cur], f.v[cur], f.w[cur]);
    return;
  }
  const int nblk = m.n_tiles + (m.nf + IB_THREADS - 1) / IB_THREADS;
  const size_t smem = m.n_tiles ? ib_tile_smem(m, sizeof(T)) : 0;
  const T* bw = reinterpret_cast<const T*>(m.bar_w);
  k_ib_interp_tiles<T><<<nblk, IB_THREADS, smem, s>>>(c, f.prm, m, fl, bw, m.bar_o, f.u[cur], f.v[cur],
                                                      f.w[cur]);
  k_ib_spread_tiles<T><<<nblk, IB_THREADS, smem, s>>>(c, m, fl, bw, m.bar_o, f.u[cur], f.v[cur], f.w[cur]);
}

template void launch_ib<double>(const Consts&, const Fields<double>&, const Markers&, const Flag&,
                                int, cudaStream_t);
template void launch_ib<float>(const Consts&, const Fields<float>&, const Markers&, const Flag&,
                               int, cudaStream_t);

}  // namespace ibm
