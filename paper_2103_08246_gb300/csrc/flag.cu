// Spring-network flag (Sec. II.B structural model), FP64, one launch per
// fluid step running all velocity-Verlet sub-steps with the fluid force held
// constant.
//
// Energies: stretching springs E = k_s/2 (|x_b - x_a| - l0)^2 on lattice edges
// and both cell diagonals; bending hinges E = k_h (1 - n_A . n_B) between the
// two triangles (of one of the two overlaid triangulations) sharing an edge.
//
// The bending force is assembled per triangle. For triangle T = (p0, p1, p2)
// with N = (p1 - p0) x (p2 - p0) and n = N / |N|, every hinge h of T with
// neighbour normal m_h contributes k_h dn/dx^T m_h, and
// dn/dx^T m = dN/dx^T (m - (n . m) n) / |N| is linear in the bracket, so
//   G_T = sum_h k_h (m_h - (n . m_h) n) / |N|,
//   f1 = (p2 - p0) x G_T,  f2 = G_T x (p1 - p0),  f0 = -(f1 + f2)
// gives the whole bending force of T on its vertices with two cross products.
//
// Each force term is written to its own slot and every vertex sums its slots
// in a fixed order (CSR list), so the result does not depend on thread
// timing. The CTAs of one thread-block cluster share the work and meet at the
// cluster barrier (hardware) between phases. Data written by other CTAs is
// read with L2-only loads.
#include <cooperative_groups.h>

#include <cmath>

#include "solver.h"

namespace cg = cooperative_groups;

namespace ibm {

struct D3 {
  double x, y, z;
};
__device__ inline D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ inline double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline D3 cross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ inline D3 ld3(const double* p, int v) {
  return {__ldcg(p + 3 * v), __ldcg(p + 3 * v + 1), __ldcg(p + 3 * v + 2)};
}
__device__ inline void st3(double* p, int q, D3 f) {
  p[3 * q] = f.x;
  p[3 * q + 1] = f.y;
  p[3 * q + 2] = f.z;
}

// 1 / sqrt(x) in FP64 from the FP32 estimate and one Newton-Raphson step for
// f(y) = 1/y^2 - x: y1 = y0 (3/2 - x y0^2 / 2). The FP32 estimate carries a
// relative error below ~2^-22, one step squares it (~1e-13), well inside the
// parity bound of the structural solve; FP64 work drops to a few multiplies.
__device__ inline double rsqrt_nr(double x) {
  const double y0 = (double)rsqrtf((float)x);
  return y0 * (1.5 - 0.5 * x * y0 * y0);
}

// unit normals of all triangles, stretching forces of all springs
__device__ void phase_normals_springs(const Flag& fl, int gt, int G) {
  for (int t = gt; t < fl.n_tri; t += G) {
    const int* tv = fl.tri + 3 * t;
    const D3 p0 = ld3(fl.X, tv[0]), p1 = ld3(fl.X, tv[1]), p2 = ld3(fl.X, tv[2]);
    const D3 N = cross(p1 - p0, p2 - p0);
    const double inv = rsqrt_nr(dot(N, N));
    st3(fl.tri_n, t, inv * N);
    fl.tri_inv[t] = inv;
  }
  const int base = 3 * fl.n_tri;
  for (int q = gt; q < fl.n_spring; q += G) {
    const int a = fl.spring[2 * q], b = fl.spring[2 * q + 1];
    const D3 d = ld3(fl.X, b) - ld3(fl.X, a);
    const double len2 = dot(d, d);
    const double il = rsqrt_nr(len2);
    const D3 f = (fl.k_s * (len2 * il - fl.l0[q]) * il) * d;   // pulls a towards b when stretched
    st3(fl.slot, base + 2 * q, f);
    st3(fl.slot, base + 2 * q + 1, -1.0 * f);
  }
}

// bending forces of every triangle from its hinges
__device__ void phase_bending(const Flag& fl, int gt, int G) {
  for (int t = gt; t < fl.n_tri; t += G) {
    const D3 n = ld3(fl.tri_n, t);
    D3 g = {0.0, 0.0, 0.0};
    for (int e = 0; e < 3; ++e) {
      const int nb = fl.tri_nb[3 * t + e];
      if (nb < 0) continue;
      const D3 m = ld3(fl.tri_n, nb);
      g = g + fl.tri_k[3 * t + e] * (m - dot(n, m) * n);
    }
    g = __ldcg(fl.tri_inv + t) * g;
    const int* tv = fl.tri + 3 * t;
    const D3 p0 = ld3(fl.X, tv[0]), p1 = ld3(fl.X, tv[1]), p2 = ld3(fl.X, tv[2]);
    const D3 f1 = cross(p2 - p0, g), f2 = cross(g, p1 - p0);
    st3(fl.slot, 3 * t, -1.0 * (f1 + f2));
    st3(fl.slot, 3 * t + 1, f1);
    st3(fl.slot, 3 * t + 2, f2);
  }
}

__device__ inline D3 gather_acc(const Flag& fl, int v) {
  D3 f = {fl.Ff[3 * v], fl.Ff[3 * v + 1], fl.Ff[3 * v + 2]};
  for (int e = fl.csr_off[v]; e < fl.csr_off[v + 1]; ++e) f = f + ld3(fl.slot, fl.csr_idx[e]);
  return fl.inv_mass[v] * f;
}

__global__ void __launch_bounds__(512) k_flag(Params* __restrict__ prm, Flag fl, int force) {
  cg::cluster_group cl = cg::this_cluster();
  if (!force && !prm->flag_pending) return;   // same value for every thread of the cluster
  const int gt = (int)cl.block_rank() * blockDim.x + threadIdx.x;
  const int G = (int)cl.num_blocks() * blockDim.x;
  const double dt = prm->flag_dt;
  const int nsub = prm->flag_nsub;
  const double hs = dt / nsub;
  phase_normals_springs(fl, gt, G);
  cl.sync();
  phase_bending(fl, gt, G);
  cl.sync();
  for (int v = gt; v < fl.nv; v += G) st3(fl.A, v, gather_acc(fl, v));
  for (int s = 0; s < nsub; ++s) {
    for (int v = gt; v < fl.nv; v += G) {
      D3 V = {fl.V[3 * v], fl.V[3 * v + 1], fl.V[3 * v + 2]};
      const D3 A = {fl.A[3 * v], fl.A[3 * v + 1], fl.A[3 * v + 2]};
      V = V + (0.5 * hs) * A;
      st3(fl.V, v, V);
      fl.X[3 * v] += hs * V.x;
      fl.X[3 * v + 1] += hs * V.y;
      fl.X[3 * v + 2] += hs * V.z;
    }
    cl.sync();
    phase_normals_springs(fl, gt, G);
    cl.sync();
    phase_bending(fl, gt, G);
    cl.sync();
    for (int v = gt; v < fl.nv; v += G) {
      const D3 a = gather_acc(fl, v);
      st3(fl.A, v, a);
      fl.V[3 * v] += 0.5 * hs * a.x;
      fl.V[3 * v + 1] += 0.5 * hs * a.y;
      fl.V[3 * v + 2] += 0.5 * hs * a.z;
    }
  }
  cl.sync();
  if (gt == 0) prm->flag_pending = 0;
}

// te_mid (3), force (3), max strain (1)
__global__ void k_flag_stats(Flag fl, double* out) {
  __shared__ double scratch[32];
  double fx = 0, fy = 0, fz = 0, st = 0;
  for (int v = threadIdx.x; v < fl.nv; v += blockDim.x) {
    fx += fl.Ff[3 * v];
    fy += fl.Ff[3 * v + 1];
    fz += fl.Ff[3 * v + 2];
  }
  for (int q = threadIdx.x; q < fl.n_spring; q += blockDim.x) {
    const int a = fl.spring[2 * q], b = fl.spring[2 * q + 1];
    const double dx = fl.X[3 * b] - fl.X[3 * a], dy = fl.X[3 * b + 1] - fl.X[3 * a + 1],
                 dz = fl.X[3 * b + 2] - fl.X[3 * a + 2];
    st = fmax(st, fabs(sqrt(dx * dx + dy * dy + dz * dz) / fl.l0[q] - 1.0));
  }
  fx = block_sum(fx, scratch);
  __syncthreads();
  fy = block_sum(fy, scratch);
  __syncthreads();
  fz = block_sum(fz, scratch);
  __syncthreads();
  st = block_max(st, scratch);
  if (threadIdx.x == 0) {
    const int te = (fl.ns - 1) * fl.nt + fl.nt / 2;
    out[0] = fl.X[3 * te];
    out[1] = fl.X[3 * te + 1];
    out[2] = fl.X[3 * te + 2];
    out[3] = fx;
    out[4] = fy;
    out[5] = fz;
    out[6] = st;
  }
}

int flag_max_cluster() {
  static int cached = -1;
  if (cached > 0) return cached;
  cudaFuncSetAttribute(k_flag, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(512);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 16;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&n, k_flag, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 8;
  }
  cached = n > 16 ? 16 : n;
  return cached;
}

void launch_flag(Params* prm, const Flag& fl, bool force, cudaStream_t s) {
  if (fl.nv == 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fl.cluster);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = fl.cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_flag, prm, fl, force ? 1 : 0);
}

void launch_flag_stats(const Flag& fl, double* out, cudaStream_t s) {
  if (fl.nv == 0) return;
  k_flag_stats<<<1, 1024, 0, s>>>(fl, out);
}

}  // namespace ibm
