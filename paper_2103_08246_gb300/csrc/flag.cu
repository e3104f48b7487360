// Spring-network flag (Sec. II.B structural model), FP64, one launch per
// fluid step running all velocity-Verlet sub-steps with the fluid force held
// constant.
//
// Energies: stretching springs E = k_s/2 (|x_b - x_a| - l0)^2 on lattice edges
// and both cell diagonals; bending hinges E = k_e (1 - n_A . n_B) between the
// two triangles (of one of the two overlaid triangulations) sharing an edge.
// Hinge force on the vertices of triangle (p0, p1, p2), N = (p1-p0) x (p2-p0):
//   g = (n_B - (n_A . n_B) n_A) / |N_A|,
//   f1 = k_e (p2 - p0) x g,  f2 = k_e g x (p1 - p0),  f0 = -(f1 + f2),
// and symmetrically for triangle B (the gradient of k_e n_A . n_B).
//
// Each force term is written to its own slot; every vertex then sums its
// slots in a fixed order (CSR list), so the result does not depend on thread
// timing. The CTAs of one thread-block cluster share the work; the cluster
// barrier separates the position update, the force evaluation and the
// gather. Positions and slots written by other CTAs are read with L2-only
// loads.
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
__device__ inline D3 ldX(const double* X, int v) {
  return {__ldcg(X + 3 * v), __ldcg(X + 3 * v + 1), __ldcg(X + 3 * v + 2)};
}
__device__ inline void stslot(double* s, int q, D3 f) {
  s[3 * q] = f.x;
  s[3 * q + 1] = f.y;
  s[3 * q + 2] = f.z;
}

__device__ void flag_forces(const Flag& fl, int gt, int G) {
  for (int q = gt; q < fl.n_spring; q += G) {
    const int a = fl.spring[2 * q], b = fl.spring[2 * q + 1];
    const D3 d = ldX(fl.X, b) - ldX(fl.X, a);
    const double len2 = dot(d, d);
    const double il = rsqrt(len2);
    const double len = len2 * il;
    const D3 f = (fl.k_s * (len - fl.l0[q]) * il) * d;   // pulls a towards b when stretched
    stslot(fl.slot, 2 * q, f);
    stslot(fl.slot, 2 * q + 1, -1.0 * f);
  }
  const int base = 2 * fl.n_spring;
  for (int q = gt; q < fl.n_hinge; q += G) {
    const int* hv = fl.hinge + 6 * q;
    const D3 a0 = ldX(fl.X, hv[0]), a1 = ldX(fl.X, hv[1]), a2 = ldX(fl.X, hv[2]);
    const D3 b0 = ldX(fl.X, hv[3]), b1 = ldX(fl.X, hv[4]), b2 = ldX(fl.X, hv[5]);
    const D3 ea1 = a1 - a0, ea2 = a2 - a0, eb1 = b1 - b0, eb2 = b2 - b0;
    const D3 NA = cross(ea1, ea2), NB = cross(eb1, eb2);
    const double ia = rsqrt(dot(NA, NA)), ib = rsqrt(dot(NB, NB));
    const D3 nA = ia * NA, nB = ib * NB;
    const double cs = dot(nA, nB);
    const double k = fl.k_hinge[q];
    const D3 gA = (k * ia) * (nB - cs * nA);
    const D3 gB = (k * ib) * (nA - cs * nB);
    const D3 fa1 = cross(ea2, gA), fa2 = cross(gA, ea1);
    const D3 fb1 = cross(eb2, gB), fb2 = cross(gB, eb1);
    const int s0 = base + 6 * q;
    stslot(fl.slot, s0 + 0, -1.0 * (fa1 + fa2));
    stslot(fl.slot, s0 + 1, fa1);
    stslot(fl.slot, s0 + 2, fa2);
    stslot(fl.slot, s0 + 3, -1.0 * (fb1 + fb2));
    stslot(fl.slot, s0 + 4, fb1);
    stslot(fl.slot, s0 + 5, fb2);
  }
}

__device__ inline D3 gather_acc(const Flag& fl, int v) {
  D3 f = {fl.Ff[3 * v], fl.Ff[3 * v + 1], fl.Ff[3 * v + 2]};
  for (int e = fl.csr_off[v]; e < fl.csr_off[v + 1]; ++e) {
    const int q = fl.csr_idx[e];
    f = f + D3{__ldcg(fl.slot + 3 * q), __ldcg(fl.slot + 3 * q + 1), __ldcg(fl.slot + 3 * q + 2)};
  }
  return fl.inv_mass[v] * f;
}

__global__ void __launch_bounds__(512) k_flag(const Params* __restrict__ prm, Flag fl) {
  cg::cluster_group cl = cg::this_cluster();
  const int gt = (int)cl.block_rank() * blockDim.x + threadIdx.x;
  const int G = (int)cl.num_blocks() * blockDim.x;
  const double dt = prm->dt;
  const int nsub = prm->n_sub;
  const double hs = dt / nsub;
  flag_forces(fl, gt, G);
  cl.sync();
  for (int v = gt; v < fl.nv; v += G) {
    const D3 a = gather_acc(fl, v);
    fl.A[3 * v] = a.x;
    fl.A[3 * v + 1] = a.y;
    fl.A[3 * v + 2] = a.z;
  }
  for (int s = 0; s < nsub; ++s) {
    for (int v = gt; v < fl.nv; v += G) {
      D3 V = {fl.V[3 * v], fl.V[3 * v + 1], fl.V[3 * v + 2]};
      const D3 A = {fl.A[3 * v], fl.A[3 * v + 1], fl.A[3 * v + 2]};
      V = V + (0.5 * hs) * A;
      fl.V[3 * v] = V.x;
      fl.V[3 * v + 1] = V.y;
      fl.V[3 * v + 2] = V.z;
      fl.X[3 * v] += hs * V.x;
      fl.X[3 * v + 1] += hs * V.y;
      fl.X[3 * v + 2] += hs * V.z;
    }
    cl.sync();
    flag_forces(fl, gt, G);
    cl.sync();
    for (int v = gt; v < fl.nv; v += G) {
      const D3 a = gather_acc(fl, v);
      fl.A[3 * v] = a.x;
      fl.A[3 * v + 1] = a.y;
      fl.A[3 * v + 2] = a.z;
      fl.V[3 * v] += 0.5 * hs * a.x;
      fl.V[3 * v + 1] += 0.5 * hs * a.y;
      fl.V[3 * v + 2] += 0.5 * hs * a.z;
    }
  }
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

void launch_flag(const Consts&, Params* prm, const Flag& fl, cudaStream_t s) {
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
  cudaLaunchKernelEx(&cfg, k_flag, (const Params*)prm, fl);
}

void launch_flag_stats(const Flag& fl, double* out, cudaStream_t s) {
  if (fl.nv == 0) return;
  k_flag_stats<<<1, 1024, 0, s>>>(fl, out);
}

}  // namespace ibm
