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
// pivots are tabulated once (FP64 arithmetic) at creation. lambda depends on
// k_y and k_z only through min(k, N - k), so the table holds the
// (N_y/2 + 1) x (N_z/2 + 1) distinct modes of every plane: a quarter of a
// field, which mostly stays in L2 between the two sweeps.
// Mode (0, 0) is singular: phi_0 = 0 is pinned, then the line mean removed,
// which sets mean(phi) = 0.
#include <cooperative_groups.h>

#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>

#include "async_copy.cuh"
#include "solver.h"

namespace ibm {

namespace cg = cooperative_groups;

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

// ---- 256-point transforms of one warp (n = 256)
// Four-step FFT, N = 8 x 32 with n = l + 32 m, k = p + 8 q: lane l holds
// z[l + 32 m], m = 0..7; an 8-point DFT over m in registers and the twiddles
// W_256^{l p} leave, for every p, a 32-point DFT over the lanes l. Those are
// split again as 32 = 8 x 4 (l = a + 4 b, q = e + 8 f): a transpose through
// the warp's shared buffer gives lane 4 p + a the values b = 0..7, an
// in-register 8-point DFT over b, twiddles W_32^{a e}, and a 4-point DFT
// across the lane quad (two shuffle stages, factors +-1 and -i only); lane
// 4 p + a then holds Z[p + 8 e + 64 f] in register e, f = brev2(a). Two real
// lines a, b travel as z = a + i b; the Hartley outputs need Z_k and Z_{N-k},
// which every lane reads back from the shared buffer for k = l + 32 t, so
// the outputs come out in the input's distribution (lane l: l + 32 t).
template <class T>
struct Cx {
  T r, i;
};
template <class T>
__device__ inline Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}

// in-register 8-point DFT: out[p] = sum_m in[m] W8^{m p}
template <class T>
__device__ inline void dft8(Cx<T> (&x)[8]) {
  const T s = (T)0.70710678118654752440;
  // radix-2 DIF stages (distance 4, 2, 1), outputs bit-reversed, then reorder
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const Cx<T> a = x[m], b = x[m + 4];
    x[m] = {a.r + b.r, a.i + b.i};
    Cx<T> d = {a.r - b.r, a.i - b.i};
    // twiddle W8^m
    if (m == 1) d = {s * (d.r + d.i), s * (d.i - d.r)};
    if (m == 2) d = {d.i, -d.r};
    if (m == 3) d = {s * (d.i - d.r), -s * (d.r + d.i)};
    x[m + 4] = d;
  }
#pragma unroll
  for (int g = 0; g < 8; g += 4)
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const Cx<T> a = x[g + m], b = x[g + m + 2];
      x[g + m] = {a.r + b.r, a.i + b.i};
      Cx<T> d = {a.r - b.r, a.i - b.i};
      if (m == 1) d = {d.i, -d.r};   // W4^1 = -i
      x[g + m + 2] = d;
    }
#pragma unroll
  for (int g = 0; g < 8; g += 2) {
    const Cx<T> a = x[g], b = x[g + 1];
    x[g] = {a.r + b.r, a.i + b.i};
    x[g + 1] = {a.r - b.r, a.i - b.i};
  }
  // bit-reversed (3 bits) -> natural order
  Cx<T> t = x[1];
  x[1] = x[4];
  x[4] = t;
  t = x[3];
  x[3] = x[6];
  x[6] = t;
}

template <class T>
__device__ inline T shfl(T v, int lane) { return __shfl_sync(0xffffffffu, v, lane); }
template <class T>
__device__ inline T shfl_x(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// Twiddles a lane needs in every transform, read once from the shared table
// tw (W_256^t = (cos, -sin)(2 pi t / 256), t = 0..255): W^{l p} after the
// 8-point DFTs, and per cross-lane stage (distance d) a sign and a factor
// that turn both halves of the butterfly into one expression,
//   lower lane: x + o = (o + x) * 1,   upper lane: (o - x) * W.
// Twiddles W^{l p} of the first pass, read once from the shared table tw
// (W_256^t = (cos, -sin)(2 pi t / 256), t = 0..255).
template <class T>
struct LaneTw {
  Cx<T> tp[8];
};

template <class T>
__device__ inline LaneTw<T> lane_twiddles(const Cx<T>* tw) {
  LaneTw<T> lt;
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < 8; ++p) lt.tp[p] = tw[(l * p) & 255];
  return lt;
}

// per-warp shared scratch: the transpose [8][36] and then Z at k + 4 (k / 64)
constexpr int WFFT_BUF = 8 * 36;
__device__ inline int zslot(int k) { return k + 4 * (k >> 6); }

template <class T>
__device__ inline void warp_hartley256(Cx<T> (&x)[8], const LaneTw<T>& lt, const Cx<T>* tw,
                                       Cx<T>* wb, T (&ha)[8], T (&hb)[8]) {
  const int l = threadIdx.x & 31;
  dft8(x);
#pragma unroll
  for (int p = 1; p < 8; ++p) x[p] = cmul(x[p], lt.tp[p]);
  // transpose: lane 4 pp + a takes Y_{a + 4 b}[pp], b = 0..7
#pragma unroll
  for (int p = 0; p < 8; ++p) wb[p * 36 + l] = x[p];
  __syncwarp();
  const int pp = l >> 2, a = l & 3;
#pragma unroll
  for (int b = 0; b < 8; ++b) x[b] = wb[pp * 36 + a + 4 * b];
  dft8(x);
#pragma unroll
  for (int e = 1; e < 8; ++e) x[e] = cmul(x[e], tw[(8 * a * e) & 255]);   // W_32^{a e}
  // 4-point DFT across the quad, decimation in frequency
  {
    const bool up = (a & 2) != 0, rot = (a & 3) == 3;
    const T sg = up ? (T)-1 : (T)1;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const Cx<T> o = {shfl_x(x[e].r, 2), shfl_x(x[e].i, 2)};
      const Cx<T> t = {o.r + sg * x[e].r, o.i + sg * x[e].i};
      x[e] = rot ? Cx<T>{t.i, -t.r} : t;   // W_4^1 = -i on the odd upper lane
    }
  }
  {
    const T sg = (a & 1) ? (T)-1 : (T)1;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const Cx<T> o = {shfl_x(x[e].r, 1), shfl_x(x[e].i, 1)};
      x[e] = {o.r + sg * x[e].r, o.i + sg * x[e].i};
    }
  }
  __syncwarp();   // the transpose has been read by every lane
  const int f = ((a & 1) << 1) | (a >> 1);
#pragma unroll
  for (int e = 0; e < 8; ++e) wb[zslot(pp + 8 * e + 64 * f)] = x[e];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int k = l + 32 * t;
    const Cx<T> zk = wb[zslot(k)], zr = wb[zslot((256 - k) & 255)];
    ha[t] = (T)0.5 * (zk.r - zk.i + zr.r + zr.i);
    hb[t] = (T)0.5 * (zk.r + zk.i - zr.r + zr.i);
  }
  __syncwarp();   // the buffer is free for the warp's next transform
}

template <class T>
__device__ inline void load_twiddles(Cx<T>* tw, const T* g) {
  for (int t = threadIdx.x; t < 128; t += blockDim.x) {
    tw[t] = {g[2 * t], g[2 * t + 1]};
    tw[t + 128] = {-g[2 * t], -g[2 * t + 1]};   // W^{t+128} = -W^t
  }
  __syncthreads();
}

// z lines (contiguous rows of 256): one warp per pair of rows, in place
template <class T>
__global__ void __launch_bounds__(256) k_dht_z256(T* __restrict__ data, int nrows, const T* __restrict__ twg) {
  __shared__ Cx<T> tw[256];
  __shared__ Cx<T> wbuf[8][WFFT_BUF];
  load_twiddles(tw, twg);
  const LaneTw<T> lt = lane_twiddles(tw);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  if (2 * warp + 1 >= nrows + 1) return;
  T* a = data + (size_t)(2 * warp) * 256;
  T* b = a + 256;
  Cx<T> x[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) x[m] = {a[l + 32 * m], b[l + 32 * m]};
  T ha[8], hb[8];
  warp_hartley256(x, lt, tw, wbuf[threadIdx.x >> 5], ha, hb);
  // lane l holds outputs l + 32 t: coalesced rows
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    a[l + 32 * t] = ha[t];
    b[l + 32 * t] = hb[t];
  }
}

// y lines (columns of a plane, ny = 256): a block stages a 256 x 32 tile
// (coalesced rows), 16 warps transform two columns each, the tile is stored back.
// Tile element (r, c) sits at r * 33 + ((c + (r >> 5)) & 31): the row pad
// spreads the column reads and writes (rows l + 32 t across the lanes) over
// the banks. Each warp's FFT scratch follows the tile in shared memory.
__device__ inline int ytile(int r, int c) { return r * 33 + ((c + (r >> 5)) & 31); }

template <class T>
__global__ void __launch_bounds__(512) k_dht_y256(T* __restrict__ data, int nz, const T* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Cx<T> tw[256];
  T* s = reinterpret_cast<T*>(smem_raw);   // [256][33]
  Cx<T>* wbuf = reinterpret_cast<Cx<T>*>(s + 256 * 33) + (threadIdx.x >> 5) * WFFT_BUF;
  const int ct = nz / 32;
  const int plane = blockIdx.x / ct, c0 = (blockIdx.x - plane * ct) * 32;
  T* base = data + (size_t)plane * 256 * nz + c0;
  for (int e = threadIdx.x; e < 256 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    s[ytile(r, c)] = base[(size_t)r * nz + c];
  }
  load_twiddles(tw, twg);   // includes __syncthreads
  const LaneTw<T> lt = lane_twiddles(tw);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  Cx<T> x[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) x[m] = {s[ytile(l + 32 * m, 2 * w)], s[ytile(l + 32 * m, 2 * w + 1)]};
  T ha[8], hb[8];
  warp_hartley256(x, lt, tw, wbuf, ha, hb);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    s[ytile(l + 32 * t, 2 * w)] = ha[t];
    s[ytile(l + 32 * t, 2 * w + 1)] = hb[t];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 256 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    base[(size_t)r * nz + c] = s[ytile(r, c)];
  }
}

// Both transforms of one 256 x 256 x-plane in a single pass: a cluster of 8
// CTAs holds the plane as eight 256 x 32 column tiles (CTA q: columns
// 32 q .. 32 q + 31). Each CTA transforms its 32 columns along y (two per
// warp per round), the cluster synchronises, then CTA q transforms rows
// 32 q .. 32 q + 31 along z (two per warp per round), gathering each row's
// eight 32-value pieces from the eight tiles through distributed shared
// memory and storing the finished rows straight to global memory. A last
// cluster barrier keeps every tile alive until all its readers are done.
// The plane is read and written once.
constexpr int DHT2D_CLUSTER = 8;
constexpr int DHT2D_THREADS = 256;
template <class T>
__global__ void __cluster_dims__(DHT2D_CLUSTER, 1, 1) __launch_bounds__(DHT2D_THREADS, sizeof(T) == 4 ? 4 : 2)
k_dht2d_256(T* __restrict__ data, const T* __restrict__ twy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Cx<T> tw[256];
  T* s = reinterpret_cast<T*>(smem_raw);   // [256][33], element (r, c) at ytile(r, c)
  Cx<T>* wbuf = reinterpret_cast<Cx<T>*>(s + 256 * 33) + (threadIdx.x >> 5) * WFFT_BUF;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int plane = blockIdx.x / DHT2D_CLUSTER;
  T* pbase = data + (size_t)plane * 256 * 256;
  {
    const T* base = pbase + 32 * q;
    constexpr int PER = 256 * 32 / DHT2D_THREADS;   // 32 values per thread
    T buf[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = threadIdx.x + t * DHT2D_THREADS;
      buf[t] = base[(size_t)(e >> 5) * 256 + (e & 31)];
    }
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = threadIdx.x + t * DHT2D_THREADS;
      s[ytile(e >> 5, e & 31)] = buf[t];
    }
  }
  load_twiddles(tw, twy);   // includes __syncthreads
  const LaneTw<T> lt = lane_twiddles(tw);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  constexpr int NW = DHT2D_THREADS / 32;
  // y: column pairs (2 cp, 2 cp + 1) of this tile
  for (int cp = w; cp < 16; cp += NW) {
    Cx<T> x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = {s[ytile(l + 32 * m, 2 * cp)], s[ytile(l + 32 * m, 2 * cp + 1)]};
    T ha[8], hb[8];
    warp_hartley256(x, lt, tw, wbuf, ha, hb);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      s[ytile(l + 32 * t, 2 * cp)] = ha[t];
      s[ytile(l + 32 * t, 2 * cp + 1)] = hb[t];
    }
  }
  cl.sync();   // every tile transformed along y (ny = nz: the same twiddles serve z)
  // z: row pairs of this CTA; value (r, k) lives in tile k / 32 at column k % 32
  for (int rp = w; rp < 16; rp += NW) {
    const int r0 = 32 * q + 2 * rp;
    Cx<T> x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const T* t = cl.map_shared_rank(s, m);
      x[m] = {t[ytile(r0, l)], t[ytile(r0 + 1, l)]};
    }
    T ha[8], hb[8];
    warp_hartley256(x, lt, tw, wbuf, ha, hb);
    // lane l holds outputs l + 32 t of both rows: coalesced rows
    T* a = pbase + (size_t)r0 * 256;
    T* b = a + 256;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      a[l + 32 * t] = ha[t];
      b[l + 32 * t] = hb[t];
    }
  }
  cl.sync();   // no tile is released while another CTA may still read it
}

// ---- FP32: both transforms of a 256 x 256 plane with thread-level radix-16
// FFTs. Four-step form N = 16 x 16 with n = j0 + 16 m, k = k1 + 16 k2:
//   Z(k1 + 16 k2) = sum_j0 W16^{j0 k2} W256^{j0 k1} sum_m z(j0 + 16 m) W16^{m k1}.
// A thread holds the 16 values m of one j0 in registers, runs the inner
// 16-point DFT there, applies W256^{j0 k1} and hands its outputs through one
// shared-memory transpose to the thread that owns k1; that thread runs the
// outer 16-point DFT over j0. No shuffles; every shared-memory access is a
// warp-contiguous row. Two real lines travel as z = a + i b and are
// separated with the Hartley identities of the file header, each thread
// producing the outputs k and N - k from the same two values.
//
// A cluster of four CTAs owns a plane (input and output planes may be the
// same or distinct). Phase y: CTA q transforms columns
// 64 q .. 64 q + 63 (complex pairs (64 q + p, 64 q + 32 + p)) along y,
// loading straight from global memory (lanes along z, coalesced), and
// stores the result in a permuted order inside the plane,
//   element (row r, column z) -> r/64 * 16384 + z/16 * 1024 + z%16 * 64 + (r/32)%2 * 32 + r%32,
// so that phase z finds its inputs (the 16 values m of one j0, for 32 row
// pairs across the lanes) as coalesced 128-byte rows. That region of the
// plane is read back from L2 at once. The permuted stores of one CTA land in
// every quarter of the plane, so in place the cluster waits until every CTA
// has consumed its phase-y loads before anyone stores (split barrier, hidden
// behind the transpose), and in every case again before phase z loads. Phase z: CTA q
// transforms rows 64 q .. 64 q + 63 (pairs (64 q + p, 64 q + 32 + p)) along
// z and stores them in natural order; the permuted block it reads is the
// block it overwrites, so no barrier follows. Plane read and written once in
// HBM; 64 bytes of shared-memory traffic per complex value.
constexpr int R16_CLUSTER = 4;
constexpr int R16_THREADS = 512;
constexpr int R16_ROW = 257;   // complex stride of the separation buffer [32][257]
constexpr size_t R16_SMEM = (size_t)32 * R16_ROW * sizeof(Cx<float>);   // >= the transpose's 16 x 16 x 32

__device__ __forceinline__ void dft4_cx(Cx<float>& a0, Cx<float>& a1, Cx<float>& a2, Cx<float>& a3) {
  const Cx<float> t0 = {a0.r + a2.r, a0.i + a2.i}, t1 = {a0.r - a2.r, a0.i - a2.i};
  const Cx<float> t2 = {a1.r + a3.r, a1.i + a3.i}, t3 = {a1.r - a3.r, a1.i - a3.i};
  a0 = {t0.r + t2.r, t0.i + t2.i};
  a2 = {t0.r - t2.r, t0.i - t2.i};
  a1 = {t1.r + t3.i, t1.i - t3.r};   // t1 - i t3
  a3 = {t1.r - t3.i, t1.i + t3.r};   // t1 + i t3
}

// (a + i b) W16^e for the exponents e = n2 k1 of the 4 x 4 split
__device__ __forceinline__ Cx<float> w16(Cx<float> a, int e) {
  const float C = 0.92387953251128675613f, S = 0.38268343236508977173f, R = 0.70710678118654752440f;
  switch (e) {
    case 1: return {a.r * C + a.i * S, a.i * C - a.r * S};
    case 2: return {(a.r + a.i) * R, (a.i - a.r) * R};
    case 3: return {a.r * S + a.i * C, a.i * S - a.r * C};
    case 4: return {a.i, -a.r};
    case 6: return {(a.i - a.r) * R, -(a.r + a.i) * R};
    case 9: return {-a.r * C - a.i * S, a.r * S - a.i * C};
    default: return a;
  }
}

// in-register 16-point DFT, natural order in and out: n = 4 n1 + n2,
// k = k1 + 4 k2, a 4-point DFT over n1, twiddles W16^{n2 k1}, a 4-point DFT
// over n2
__device__ __forceinline__ void dft16(Cx<float> (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4_cx(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2) x[4 * k1 + n2] = w16(x[4 * k1 + n2], n2 * k1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4_cx(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // slot 4 k1 + k2 holds Z(k1 + 4 k2): transpose the 4 x 4 index
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a + 1; b < 4; ++b) {
      const Cx<float> t = x[4 * a + b];
      x[4 * a + b] = x[4 * b + a];
      x[4 * b + a] = t;
    }
}

__device__ __forceinline__ int r16_perm(int row, int z) {
  return (row >> 6) * 16384 + (z >> 4) * 1024 + (z & 15) * 64 + ((row >> 5) & 1) * 32 + (row & 31);
}

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Inner DFT of the thread's 16 values, the W256^{j0 k1} twiddles, the
// transpose, and the outer DFT: on return x[k2] = Z(k1 + 16 k2) of the lane's
// line pair, k1 = the warp index. `pre_wait` runs between the transpose's
// stores and loads (the cluster arrive of phase y).
template <class F>
__device__ __forceinline__ void r16_fft(Cx<float> (&x)[16], const Cx<float>* tw, Cx<float>* buf, int w, int l,
                                        F pre_wait) {
  dft16(x);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) buf[(k1 * 16 + w) * 32 + l] = k1 ? cmul(x[k1], tw[w * k1]) : x[0];   // w k1 <= 225
  pre_wait();
  __syncthreads();
#pragma unroll
  for (int j0 = 0; j0 < 16; ++j0) x[j0] = buf[(w * 16 + j0) * 32 + l];
  dft16(x);
  __syncthreads();   // the transpose buffer is free for the separation buffer
}

__global__ void __cluster_dims__(R16_CLUSTER, 1, 1) __launch_bounds__(R16_THREADS, 2)
k_dht2d_r16(const float* in, float* out, const float* __restrict__ twy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Cx<float> tw[256];
  Cx<float>* buf = reinterpret_cast<Cx<float>*>(smem_raw);
  const int q = (int)(blockIdx.x % R16_CLUSTER);   // rank in the cluster (clusters are consecutive blocks)
  const size_t plane = (size_t)(blockIdx.x / R16_CLUSTER) * 65536;
  float* P = out + plane;
  const bool inplace = in == out;   // the same for the whole grid
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  Cx<float> x[16];
  // ---- phase y: columns (64 q + l, 64 q + 32 + l), rows w + 16 m
  {
    const float* col = in + plane + 64 * q + l;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int r = w + 16 * m;
      x[m] = {__ldcg(col + r * 256), __ldcg(col + r * 256 + 32)};
    }
  }
  load_twiddles(tw, twy);   // includes __syncthreads
  r16_fft(x, tw, buf, w, l, [inplace] {
    if (inplace) cluster_arrive_release();   // every phase-y load consumed
  });
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) buf[l * R16_ROW + w + 16 * k2] = x[k2];
  __syncthreads();
  if (inplace) cluster_wait_acquire();   // no CTA still needs an original value of this plane
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const int p = 2 * w + pp;
    const Cx<float>* Zp = buf + p * R16_ROW;
    const int za = 64 * q + p, zb = za + 32;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int k = l + 32 * v;
      const int kr = k == 0 ? 128 : 256 - k;   // k = 0 and 128 are their own mirrors
      const Cx<float> zk = Zp[k], zr = Zp[kr];
      const Cx<float> mk = k == 0 ? zk : zr, mr = k == 0 ? zr : zk;
      P[r16_perm(k, za)] = 0.5f * (zk.r - zk.i + mk.r + mk.i);
      P[r16_perm(k, zb)] = 0.5f * (zk.r + zk.i - mk.r + mk.i);
      P[r16_perm(kr, za)] = 0.5f * (zr.r - zr.i + mr.r + mr.i);
      P[r16_perm(kr, zb)] = 0.5f * (zr.r + zr.i - mr.r + mr.i);
    }
  }
  cluster_arrive_release();
  cluster_wait_acquire();   // the whole plane holds the y transform (permuted)
  // ---- phase z: rows (64 q + l, 64 q + 32 + l), columns w + 16 m
  {
    const float* blk = P + q * 16384 + w * 64 + l;
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = {__ldcg(blk + m * 1024), __ldcg(blk + m * 1024 + 32)};
  }
  r16_fft(x, tw, buf, w, l, [] {});
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) buf[l * R16_ROW + w + 16 * k2] = x[k2];
  __syncthreads();
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const int p = 2 * w + pp;
    const Cx<float>* Zp = buf + p * R16_ROW;
    float* ra = P + (size_t)(64 * q + p) * 256;
    float* rb = ra + 32 * 256;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int k = l + 32 * v;
      const int kr = k == 0 ? 128 : 256 - k;
      const Cx<float> zk = Zp[k], zr = Zp[kr];
      const Cx<float> mk = k == 0 ? zk : zr, mr = k == 0 ? zr : zk;
      ra[k] = 0.5f * (zk.r - zk.i + mk.r + mk.i);
      rb[k] = 0.5f * (zk.r + zk.i - mk.r + mk.i);
      ra[kr] = 0.5f * (zr.r - zr.i + mr.r + mr.i);
      rb[kr] = 0.5f * (zr.r + zr.i - mr.r + mr.i);
    }
  }
}

// Thomas solve along x per mode; rhs scaled by h^2 / (ny nz) (Hartley
// normalisation). One thread per mode walks x (coalesced across modes) in
// chunks of PF planes; the loads of the next chunk (right-hand side and
// inverse pivots) are issued before the current chunk's recursion, so each
// thread keeps up to 4 PF independent loads in flight. Past the row from
// which a mode's stored pivots equal their limit (a few rows for all but
// the lowest modes) the limit stays in a register and the chunks carry
// right-hand sides only, twice as many per chunk in FP32.
constexpr int PF = 16;
__host__ __device__ inline size_t ptab_plane(const Consts& c) {
  return (size_t)(c.ny / 2 + 1) * (c.nz / 2 + 1);
}
__device__ inline size_t ptab_index(const Consts& c, int jk) {
  const int ky = jk / c.nz, kz = jk - ky * c.nz;
  const int qy = ky <= c.ny / 2 ? ky : c.ny - ky, qz = kz <= c.nz / 2 ? kz : c.nz - kz;
  return (size_t)qy * (c.nz / 2 + 1) + qz;
}

// storage conversions: FP32 / FP64 fields, or bfloat16 (the mixed solve's correction)
template <class T, class S>
__device__ inline T from_store(S v) {
  if constexpr (std::is_same<S, __nv_bfloat16>::value) return __bfloat162float(v);
  else return (T)v;
}
template <class S, class T>
__device__ inline S to_store(T v) {
  if constexpr (std::is_same<S, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
  else return (S)v;
}

// forward elimination over planes [i0, i1) in chunks of N planes, the next
// chunk's loads issued before the current chunk's recursion (two chunks in
// flight); TAB: inverse pivots from the table, else the converged limit
template <int N, bool TAB, class T, class LDF, class STF>
__device__ __forceinline__ void px_forward(LDF LD, STF ST, const T* iv, size_t PT, int P, T lim, T scale,
                                           bool zero_mode, int i0, int i1, T& y) {
  constexpr int NT = TAB ? N : 1;
  const int nch = (i1 - i0) / N;
  T rd[N], rt[NT];
  if (nch > 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      rd[q] = LD((size_t)(i0 + q) * P);
      if constexpr (TAB) rt[q] = iv[(size_t)(i0 + q) * PT];
    }
  }
  int i = i0;
  for (int ch = 0; ch < nch; ++ch, i += N) {
    T nd[N], nt[NT];
    if (ch + 1 < nch) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        nd[q] = LD((size_t)(i + N + q) * P);
        if constexpr (TAB) nt[q] = iv[(size_t)(i + N + q) * PT];
      }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if constexpr (TAB) {
        const T rhs = (zero_mode && i + q == 0) ? (T)0 : rd[q] * scale;
        y = (rhs - y) * rt[q];
      } else {
        y = (rd[q] * scale - y) * lim;
      }
      ST((size_t)(i + q) * P, y);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      rd[q] = nd[q];
      if constexpr (TAB) rt[q] = nt[q];
    }
  }
  for (; i < i1; ++i) {   // the partial chunk
    const size_t o = (size_t)i * P;
    if constexpr (TAB) {
      const T rhs = (zero_mode && i == 0) ? (T)0 : LD(o) * scale;
      y = (rhs - y) * iv[(size_t)i * PT];
    } else {
      y = (LD(o) * scale - y) * lim;
    }
    ST(o, y);
  }
}

// back substitution over planes i1 - 1 down to i0 (x holds x_{i1} on entry),
// the partial chunk first, then chunks of N as above; the line sum of mode
// (0, 0) gathered on the way
template <int N, bool TAB, class T, class LDF, class STF>
__device__ __forceinline__ void px_backward(LDF LD, STF ST, const T* iv, size_t PT, int P, T lim, bool zero_mode,
                                            int i0, int i1, T& x, T& lsum) {
  constexpr int NT = TAB ? N : 1;
  int i = i1 - 1;
  const int rem = (i1 - i0) % N;
  for (int r = 0; r < rem; ++r, --i) {
    const size_t o = (size_t)i * P;
    T cp = lim;
    if constexpr (TAB) cp = (zero_mode && i == 0) ? (T)0 : iv[(size_t)i * PT];
    x = LD(o) - cp * x;
    ST(o, x);
    lsum += x;
  }
  const int nch = (i1 - i0) / N;   // full chunks below: planes i, i - 1, ..., i0
  T rd[N], rt[NT];
  if (nch > 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      rd[q] = LD((size_t)(i - q) * P);
      if constexpr (TAB) rt[q] = iv[(size_t)(i - q) * PT];
    }
  }
  for (int ch = 0; ch < nch; ++ch, i -= N) {
    T nd[N], nt[NT];
    if (ch + 1 < nch) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        nd[q] = LD((size_t)(i - N - q) * P);
        if constexpr (TAB) nt[q] = iv[(size_t)(i - N - q) * PT];
      }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T cp = lim;
      if constexpr (TAB) cp = (zero_mode && i - q == 0) ? (T)0 : rt[q];
      x = rd[q] - cp * x;
      ST((size_t)(i - q) * P, x);
      lsum += x;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      rd[q] = nd[q];
      if constexpr (TAB) rt[q] = nt[q];
    }
  }
}

// Single pass over the converged rows of modes whose converged inverse pivot
// is at most 1/2 in magnitude (FP32 arithmetic): there the back substitution
// x_j = y_j - lim x_{j+1} equals sum_k (-lim)^k y_{j+k}, and the sum after
// PW terms is below lim^PW <= 2^-24 of x, the FP32 rounding. Each chunk of PW
// rows is emitted once the next chunk's forward values exist: its last row
// from the truncated sum, the others by the exact recursion downward. The
// forward values of those rows never go to memory (read once, written once
// instead of read, written, read, written). Rows below ia (table pivots) and
// the last chunk with the remaining rows keep the stored forward values and
// the exact back substitution.
constexpr int PW = 24;
template <class T, class LDF, class STF>
__device__ __forceinline__ void px_single(LDF LD, STF ST, const T* iv, size_t PT, int P, T lim, T scale, int ia,
                                          int nx) {
  T y = 0;
  for (int i = 0; i < ia; ++i) {   // head: table pivots, forward values stored
    const size_t o = (size_t)i * P;
    y = (LD(o) * scale - y) * iv[(size_t)i * PT];
    ST(o, y);
  }
  const int nch = (nx - 1 - ia) / PW;   // >= 1 (checked by the caller)
  T yc[PW], yp[PW], nd[PW];
#pragma unroll
  for (int q = 0; q < PW; ++q) nd[q] = LD((size_t)(ia + q) * P);
  T x_ia = 0;
  for (int ch = 0; ch < nch; ++ch) {
    const int i0 = ia + ch * PW;
#pragma unroll
    for (int q = 0; q < PW; ++q) yp[q] = yc[q];
#pragma unroll
    for (int q = 0; q < PW; ++q) yc[q] = nd[q];
    if (ch + 1 < nch) {
#pragma unroll
      for (int q = 0; q < PW; ++q) nd[q] = LD((size_t)(i0 + PW + q) * P);
    }
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      y = (yc[q] * scale - y) * lim;
      yc[q] = y;
    }
    if (ch > 0) {   // emit the previous chunk
      T acc = yc[PW - 2];
#pragma unroll
      for (int k = PW - 3; k >= 0; --k) acc = yc[k] - lim * acc;
      T x = yp[PW - 1] - lim * acc;
      const int j0 = i0 - PW;
      ST((size_t)(j0 + PW - 1) * P, x);
#pragma unroll
      for (int q = PW - 2; q >= 0; --q) {
        x = yp[q] - lim * x;
        ST((size_t)(j0 + q) * P, x);
      }
      if (ch == 1) x_ia = x;
    }
  }
  // tail: the last chunk's forward values, the remaining rows and the last
  // row (its own pivot) stored; exact back substitution down to the last chunk
  const int it = ia + (nch - 1) * PW;
#pragma unroll
  for (int q = 0; q < PW; ++q) ST((size_t)(it + q) * P, yc[q]);
  for (int i = it + PW; i < nx - 1; ++i) {
    const size_t o = (size_t)i * P;
    y = (LD(o) * scale - y) * lim;
    ST(o, y);
  }
  {
    const size_t o = (size_t)(nx - 1) * P;
    y = (LD(o) * scale - y) * iv[(size_t)(nx - 1) * PT];
    ST(o, y);
  }
  T x = y;
  for (int i = nx - 2; i >= it; --i) {
    const size_t o = (size_t)i * P;
    x = LD(o) - lim * x;
    ST(o, x);
  }
  if (nch == 1) x_ia = x;
  x = x_ia;   // head: exact back substitution with the table pivots
  for (int i = ia - 1; i >= 0; --i) {
    const size_t o = (size_t)i * P;
    x = LD(o) - iv[(size_t)i * PT] * x;
    ST(o, x);
  }
}

template <class T, class S>
__global__ void __launch_bounds__(128) k_poisson_x(Consts c, const T* __restrict__ tab, const int* __restrict__ conv,
                                                   S* __restrict__ phi, T scale, double* __restrict__ mean00) {
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  const int nx = c.nx;
  S* d = phi + jk;
  auto LD = [d](size_t o) { return from_store<T>(d[o]); };
  auto ST = [d](size_t o, T v) { d[o] = to_store<S>(v); };
  const size_t mi = ptab_index(c, jk);
  const T* iv = tab + mi;
  const size_t PT = ptab_plane(c);
  const bool zero_mode = (jk == 0);
  // planes [0, ia) take the table's pivots, [ia, nx - 1) the converged
  // limit held in a register (bitwise the table's values there), plane
  // nx - 1 its own; ia is the largest convergence row of the warp's modes,
  // so the split is warp-uniform and the converged range spends every load
  // slot on the right-hand side (chunks of PB planes)
  const int ia = min(max(__reduce_max_sync(__activemask(), conv[mi]), 1), nx - 1);
  const T lim = iv[(size_t)(nx - 2) * PT];
  if constexpr (sizeof(T) == 4) {
    // every mode of the warp decays fast enough for the single pass (never mode (0, 0))
    if (nx - 1 - ia >= PW && __all_sync(__activemask(), fabsf(lim) <= 0.5f) && !zero_mode) {
      px_single<T>(LD, ST, iv, PT, P, lim, scale, ia, nx);
      return;
    }
  }
  constexpr int PB = sizeof(T) == 8 ? PF : 2 * PF;
  T y = 0;
  px_forward<PF, true>(LD, ST, iv, PT, P, lim, scale, zero_mode, 0, ia, y);
  px_forward<PB, false>(LD, ST, iv, PT, P, lim, scale, zero_mode, ia, nx - 1, y);
  {
    const size_t o = (size_t)(nx - 1) * P;
    y = (LD(o) * scale - y) * iv[(size_t)(nx - 1) * PT];
    ST(o, y);
  }
  // back substitution from the top (in T: an FP64 conversion per plane and
  // mode would load the narrow FP64 pipe)
  T x = y;  // x_{nx-1} = dp_{nx-1}
  T lsum = x;
  px_backward<PB, false>(LD, ST, iv, PT, P, lim, zero_mode, ia, nx - 1, x, lsum);
  px_backward<PF, true>(LD, ST, iv, PT, P, lim, zero_mode, 0, ia, x, lsum);
  // the mean is removed by k_mode00_sub, in parallel over the planes
  if (zero_mode) *mean00 = (double)lsum / nx;
}

// gauge mean(phi) = 0: subtract the line mean of mode (0, 0) in every plane
template <class S>
__global__ void k_mode00_sub(Consts c, S* __restrict__ phi, const double* __restrict__ mean00) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < c.nx) {
    S& v = phi[(size_t)i * c.ny * c.nz];
    v = to_store<S>(from_store<double>(v) - *mean00);
  }
}

// inverse pivots 1 / (diag_i - c'_{i-1}) of every distinct mode, FP64 arithmetic
template <class T>
__global__ void k_poisson_table(Consts c, T* __restrict__ tab, int* __restrict__ conv) {
  const int qz_n = c.nz / 2 + 1;
  const int PT = (c.ny / 2 + 1) * qz_n;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= PT) return;
  const int ky = m / qz_n, kz = m - ky * qz_n;
  const double sy = sin(M_PI * ky / c.ny), sz = sin(M_PI * kz / c.nz);
  const double lam = -4.0 * sy * sy - 4.0 * sz * sz;
  const bool pinned = (m == 0);
  const int nx = c.nx;
  double cp = 0.0;
  for (int i = 0; i < nx; ++i) {
    double diag = (i == 0 || i == nx - 1) ? -1.0 + lam : -2.0 + lam;
    double lower = i == 0 ? 0.0 : 1.0;
    if (pinned && i == 0) diag = 1.0;              // pinned phi_0 = 0
    const double prev_cp = (pinned && i == 1) ? 0.0 : cp;
    const double denom = diag - lower * prev_cp;
    const double inv = 1.0 / denom;
    tab[(size_t)i * PT + m] = (T)inv;
    cp = inv;  // upper = 1
  }
  // rows 1 .. nx - 2 share one recursion whose pivots converge to a limit;
  // the first row from which the stored pivots equal the stored limit
  const T lim = tab[(size_t)(nx - 2) * PT + m];
  int ic = nx - 2;
  while (ic > 0 && tab[(size_t)(ic - 1) * PT + m] == lim) --ic;
  conv[m] = ic;
}

template <class T>
void launch_dht_y(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  if (c.ny == 256 && c.nz % 32 == 0) {
    const size_t sh = (size_t)256 * 33 * sizeof(T) + 16 * WFFT_BUF * sizeof(Cx<T>);
    k_dht_y256<T><<<c.nx * (c.nz / 32), 512, sh, s>>>(f.phi, c.nz, f.tw_y);
    return;
  }
  const int n = c.ny, logn = (int)std::lround(std::log2((double)n));
  const int W = c.nz < 16 ? c.nz : 16;
  const size_t sh = (size_t)(W / 2) * n * sizeof(typename Vec2<T>::type);
  // group = one x plane; lines = nz columns; positions nz apart
  k_dht<T, false><<<c.nx * (c.nz / W), 256, sh, s>>>(f.phi, n, logn, W, c.nz, plane(c),
                                                       (size_t)c.nz, f.tw_y);
}

template <class T>
void launch_dht_z(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  if (c.nz == 256) {
    const int rows = c.nx * c.ny;   // even: ny is an even power of two
    k_dht_z256<T><<<(rows / 2 + 7) / 8, 256, 0, s>>>(f.phi, rows, f.tw_z);
    return;
  }
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

  k_poisson_x<T, T><<<(P + 127) / 128, 128, 0, s>>>(c, f.ptab, f.pconv, buf, scale, f.mean00);
  k_mode00_sub<T><<<(c.nx + 255) / 256, 256, 0, s>>>(c, buf, f.mean00);
}

// the same on bfloat16 storage (FP32 arithmetic)
void launch_poisson_x_bf16(const Consts& c, const Fields<float>& f, void* buf, cudaStream_t s) {
  const int P = c.ny * c.nz;
  const float scale = (float)(c.h * c.h / ((double)c.ny * c.nz));
  __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(buf);
  k_poisson_x<float, __nv_bfloat16><<<(P + 127) / 128, 128, 0, s>>>(c, f.ptab, f.pconv, b, scale, f.mean00);
  k_mode00_sub<__nv_bfloat16><<<(c.nx + 255) / 256, 256, 0, s>>>(c, b, f.mean00);
}

template <class T>
void launch_poisson_x(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  launch_poisson_x_on(c, f, f.phi, s);
}

template <class T>
bool launch_dht2d(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  if (c.ny != 256 || c.nz != 256) return false;
  if constexpr (sizeof(T) == 4) {
    k_dht2d_r16<<<c.nx * R16_CLUSTER, R16_THREADS, R16_SMEM, s>>>(f.phi, f.phi, f.tw_y);
    return true;
  }
  const size_t sh = (size_t)256 * 33 * sizeof(T) + (DHT2D_THREADS / 32) * WFFT_BUF * sizeof(Cx<T>);
  k_dht2d_256<T><<<c.nx * DHT2D_CLUSTER, DHT2D_THREADS, sh, s>>>(f.phi, f.tw_y);
  return true;
}

bool launch_dht2d_on(const Consts& c, const Fields<float>& f, const float* in, float* out, cudaStream_t s) {
  if (c.ny != 256 || c.nz != 256) return false;
  k_dht2d_r16<<<c.nx * R16_CLUSTER, R16_THREADS, R16_SMEM, s>>>(in, out, f.tw_y);
  return true;
}

// the same transform of `nplanes` 256 x 256 planes outside a solver state
// (the generator's spectral relaxation); tw: the 256-point twiddles
bool dht2d_planes_fp32(const float* in, float* out, int nplanes, const float* tw, cudaStream_t s) {
  if (nplanes <= 0) return true;
  k_dht2d_r16<<<nplanes * R16_CLUSTER, R16_THREADS, R16_SMEM, s>>>(in, out, tw);
  return cudaGetLastError() == cudaSuccess;
}

template <class T>
void launch_poisson(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  if (launch_dht2d(c, f, s)) {
    launch_poisson_x(c, f, s);
    launch_dht2d(c, f, s);
    return;
  }
  launch_dht_y(c, f, s);
  launch_dht_z(c, f, s);
  launch_poisson_x(c, f, s);
  launch_dht_z(c, f, s);
  launch_dht_y(c, f, s);
}

size_t poisson_table_size(const Consts& c) { return (size_t)c.nx * ptab_plane(c); }
size_t poisson_modes(const Consts& c) { return ptab_plane(c); }

template <class T>
void launch_poisson_table(const Consts& c, const Fields<T>& f, cudaStream_t s) {
  const int PT = (int)ptab_plane(c);
  k_poisson_table<T><<<(PT + 127) / 128, 128, 0, s>>>(c, f.ptab, f.pconv);
}

template void launch_poisson<double>(const Consts&, const Fields<double>&, cudaStream_t);
template bool launch_dht2d<double>(const Consts&, const Fields<double>&, cudaStream_t);
template bool launch_dht2d<float>(const Consts&, const Fields<float>&, cudaStream_t);
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
  cudaFuncSetAttribute(k_dht2d_256<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht2d_256<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht2d_r16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R16_SMEM);
  cudaFuncSetAttribute(k_dht_y256<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht_y256<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_dht<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace ibm
