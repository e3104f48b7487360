// Pressure Poisson equation L_h phi = D (Sec. II.B projection step): transforms
// in the periodic y and z directions, one tridiagonal (Thomas) solve along x
// per transverse wavenumber pair, inverse transforms.
//
// Transform: the discrete Hartley transform H x (k) = sum_j x_j cas(2 pi j k / N),
// cas = cos + sin. The periodic second difference is symmetric and circulant,
// so its eigenvalue lambda(k) = (2 cos(2 pi k / N) - 2) / h^2 is shared by
// cos and sin modes; the separable 2-D Hartley transform H_y H_z therefore
// diagonalises the y-z part of L_h exactly like the DFT, while every array
// stays real. H is its own inverse up to 1/N. Two real lines are packed into
// one complex FFT (radix-2, decimation in time, in shared memory) and
// separated afterwards:
//   Z = FFT(a + i b):  H a (k) = (Re Z_k - Im Z_k + Re Z_{N-k} + Im Z_{N-k}) / 2
//                      H b (k) = (Re Z_k + Im Z_k - Re Z_{N-k} + Im Z_{N-k}) / 2
//
// x solve, with the equation scaled by h^2 (Neumann ends phi_{-1} = phi_0,
// phi_nx = phi_{nx-1}):
//   phi_{i-1} + (-2 + lambda h^2) phi_i + phi_{i+1} = h^2 D_i,
// lambda h^2 = -4 sin^2(pi k_y / N_y) - 4 sin^2(pi k_z / N_z). The LU inverse
// pivots of every mode are tabulated once (FP64 arithmetic) at creation.
// Mode (0, 0) is singular: phi_0 = 0 is pinned, then the line mean removed,
// which sets mean(phi) = 0.
#include <cmath>

#include "solver.h"

namespace ibm {

__device__ inline int bitrev(int x, int logn) { return (int)(__brev((unsigned)x) >> (32 - logn)); }

// Transform W real lines of length n held in `data` (global), in place.
// CONTIG: lines are contiguous (z) with consecutive lines nz apart;
// otherwise positions are `pstride` apart and consecutive lines adjacent (y).
template <class T, bool CONTIG>
__global__ void __launch_bounds__(256)
k_dht(T* __restrict__ data, int n, int logn, int W, int lines_per_group, size_t group_stride,
      size_t pstride, const T* __restrict__ tw) {
  using C2 = typename Vec2<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C2* Z = reinterpret_cast<C2*>(smem_raw);   // [W/2][n]
  const int groups_per_outer = lines_per_group / W;
  const int outer = blockIdx.x / groups_per_outer;
  const int g = blockIdx.x - outer * groups_per_outer;
  T* base = data + (size_t)outer * group_stride + (size_t)g * W * (CONTIG ? (size_t)n : (size_t)1);
  const int tot = W * n;
  // load with bit reversal, pairing lines (2q, 2q+1) as (re, im) of complex line q
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int l, j;
    size_t gi;
    if (CONTIG) {
      l = e / n;
      j = e - l * n;
      gi = (size_t)l * n + j;
    } else {
      j = e / W;
      l = e - j * W;
      gi = (size_t)j * pstride + l;
    }
    const T val = base[gi];
    C2* zz = Z + (size_t)(l >> 1) * n + bitrev(j, logn);
    if (l & 1) zz->y = val; else zz->x = val;
  }
  __syncthreads();
  const int half = n >> 1;
  const int nb = (W >> 1) * half;
  for (int m = 1; m < n; m <<= 1) {
    const int tstep = n / (2 * m);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      const int q = t / half;
      const int b = t - q * half;
      const int pos = b & (m - 1);
      const int i1 = ((b - pos) << 1) + pos;
      const int i2 = i1 + m;
      C2* zq = Z + (size_t)q * n;
      const C2 wv = reinterpret_cast<const C2*>(tw)[pos * tstep];
      const C2 a = zq[i1], c = zq[i2];
      const T br = c.x * wv.x - c.y * wv.y;
      const T bi = c.x * wv.y + c.y * wv.x;
      zq[i1] = C2{a.x + br, a.y + bi};
      zq[i2] = C2{a.x - br, a.y - bi};
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int l, j;
    size_t gi;
    if (CONTIG) {
      l = e / n;
      j = e - l * n;
      gi = (size_t)l * n + j;
    } else {
      j = e / W;
      l = e - j * W;
      gi = (size_t)j * pstride + l;
    }
    const C2* zq = Z + (size_t)(l >> 1) * n;
    const C2 zk = zq[j];
    const C2 zr = zq[j == 0 ? 0 : n - j];
    const T hv = (l & 1) ? (zk.x + zk.y - zr.x + zr.y) : (zk.x - zk.y + zr.x + zr.y);
    base[gi] = (T)0.5 * hv;
  }
}

// Thomas solve along x per mode; rhs scaled by h^2 / (ny nz) (Hartley normalisation).
template <class T>
__global__ void k_poisson_x(Consts c, const T* __restrict__ tab, T* __restrict__ phi, T scale) {
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  const int nx = c.nx;
  T* d = phi + jk;
  const T* iv = tab + jk;
  const bool zero_mode = (jk == 0);
  T y = 0;
  for (int i = 0; i < nx; ++i) {
    const size_t o = (size_t)i * P;
    T rhs = (zero_mode && i == 0) ? (T)0 : d[o] * scale;
    y = (rhs - y) * iv[o];
    d[o] = y;
  }
  T x = y;  // x_{nx-1} = dp_{nx-1}
  for (int i = nx - 2; i >= 0; --i) {
    const size_t o = (size_t)i * P;
    const T cp = (zero_mode && i == 0) ? (T)0 : iv[o];
    x = d[o] - cp * x;
    d[o] = x;
  }
  if (zero_mode) {
    double s = 0.0;
    for (int i = 0; i < nx; ++i) s += (double)d[(size_t)i * P];
    const T mean = (T)(s / nx);
    for (int i = 0; i < nx; ++i) d[(size_t)i * P] -= mean;
  }
}

// inverse pivots 1 / (diag_i - c'_{i-1}) of every mode, FP64 arithmetic
template <class T>
__global__ void k_poisson_table(Consts c, T* __restrict__ tab) {
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  const int ky = jk / c.nz, kz = jk - ky * c.nz;
  const double sy = sin(M_PI * ky / c.ny), sz = sin(M_PI * kz / c.nz);
  const double lam = -4.0 * sy * sy - 4.0 * sz * sz;
  const int nx = c.nx;
  double cp = 0.0;
  for (int i = 0; i < nx; ++i) {
    double diag = (i == 0 || i == nx - 1) ? -1.0 + lam : -2.0 + lam;
    double lower = i == 0 ? 0.0 : 1.0;
    if (jk == 0 && i == 0) diag = 1.0;              // pinned phi_0 = 0
    const double prev_cp = (jk == 0 && i == 1) ? 0.0 : cp;
    const double denom = diag - lower * prev_cp;
    const double inv = 1.0 / denom;
    tab[(size_t)i * P + jk] = (T)inv;
    cp = inv;  // upper = 1
  }
}

template <class T>
void launch_dht_y(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const int n = c.ny, logn = (int)std::lround(std::log2((double)n));
  const int W = c.nz < 16 ? c.nz : 16;
  const size_t sh = (size_t)(W / 2) * n * sizeof(typename Vec2<T>::type);
  // group = one x plane; lines = nz columns; positions nz apart
  k_dht<T, false><<<c.nx * (c.nz / W), 256, sh, s>>>(f.phi, n, logn, W, c.nz, plane(c),
                                                       (size_t)c.nz, f.tw_y);
}

template <class T>
void launch_dht_z(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const int n = c.nz, logn = (int)std::lround(std::log2((double)n));
  const int lines = c.nx * c.ny;
  int W = 16;
  while (lines % W) W >>= 1;   // ny is an even power of two, so W >= 2
  const size_t sh = (size_t)(W / 2) * n * sizeof(typename Vec2<T>::type);
  k_dht<T, true><<<lines / W, 256, sh, s>>>(f.phi, n, logn, W, lines, 0, 1, f.tw_z);
}

template <class T>
void launch_poisson_x_on(const Consts& c, const Fields<T>& f, T* buf, cudaStream_t s) {
  const int P = c.ny * c.nz;
  const T scale = (T)(c.h * c.h / ((double)c.ny * c.nz));
  k_poisson_x<T><<<(P + 127) / 128, 128, 0, s>>>(c, f.ptab, buf, scale);
}

template <class T>
void launch_poisson_x(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  launch_poisson_x_on(c, f, f.phi, s);
}

template <class T>
void launch_poisson(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  launch_dht_y(c, f, s);
  launch_dht_z(c, f, s);
  launch_poisson_x(c, f, s);
  launch_dht_z(c, f, s);
  launch_dht_y(c, f, s);
}

template <class T>
void launch_poisson_table(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const int P = c.ny * c.nz;
  k_poisson_table<T><<<(P + 127) / 128, 128, 0, s>>>(c, f.ptab);
}

template void launch_poisson<double>(const Consts&, const Fields<double>&, cudaStream_t);
template void launch_dht_y<double>(const Consts&, const Fields<double>&, cudaStream_t);
template void launch_dht_y<float>(const Consts&, const Fields<float>&, cudaStream_t);
template void launch_dht_z<double>(const Consts&, const Fields<double>&, cudaStream_t);
template void launch_dht_z<float>(const Consts&, const Fields<float>&, cudaStream_t);
template void launch_poisson_x<double>(const Consts&, const Fields<double>&, cudaStream_t);
template void launch_poisson_x_on<float>(const Consts&, const Fields<float>&, float*, cudaStream_t);
template void launch_poisson_x_on<double>(const Consts&, const Fields<double>&, double*, cudaStream_t);
template void launch_poisson_x<float>(const Consts&, const Fields<float>&, cudaStream_t);
template void launch_poisson<float>(const Consts&, const Fields<float>&, cudaStream_t);
template void launch_poisson_table<double>(const Consts&, const Fields<double>&, cudaStream_t);
template void launch_poisson_table<float>(const Consts&, const Fields<float>&, cudaStream_t);

// opt in to large dynamic shared memory for the transform kernels
void poisson_set_attributes() {
  cudaFuncSetAttribute(k_dht<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace ibm
