// Shared device-side definitions of the solver library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace ibm {

// Per-step scalars kept in device memory, so that a captured step graph can
// run with a time step computed on the device (CFL mode).
struct Params {
  double dt;          // current step
  double dt_old;      // previous step (AB2 weights)
  double alpha, beta; // AB2 weights
  double r;           // nu * dt / (2 h^2), implicit diffusion number
  double t;           // time at the start of the step
  double mass_shift;  // added to u on the outflow face (mass fix)
  double q_in, q_out; // volume fluxes (last mass fix)
  double speed_max;   // max_cells(|u|+|v|+|w|) of the current velocity
  double slip_max;    // max |U* - U| over markers of the last forcing
  double dt_fixed;    // > 0: fixed step; otherwise CFL mode
  double cfl;         // Courant number in CFL mode
  long long step;     // steps done
  int n_sub;          // structural sub-steps of the current step
  int first;          // 1 until the first step has run (Euler start)
  int error;          // bit mask of device-side errors
  int flag_nsub;      // sub-steps of the pending structural update
  double flag_dt;     // fluid step of the pending structural update
  int flag_pending;   // 1 after a forcing step until the flag has been advanced
  int af_h;           // warm-up length of the segmented implicit line solves
  double af_rho;      // exp(-theta) of the implicit factors
  // FP32 copies of the per-step scalars, written once per step, so that FP32
  // kernels never convert from FP64 per thread (conversions run on the FP64
  // pipe)
  float f_dt, f_alpha, f_beta, f_r, f_ir, f_rho, f_mass_shift;
  float f_gdt;        // dt / h
  float f_hnu;        // nu dt / (2 h^2)
  float f_cc;         // U dt / h
  float f_sc_div;     // 1 / (h dt)
};

// Host-provided constants of a problem.
struct Consts {
  int nx, ny, nz;
  double h, inv_h, nu, lx, ly, lz;
  double u_in;        // inflow speed U
  double omega_max;   // structural stiffness bound (sub-step count)
  int rhs_planes;     // tile: x planes per block of the streamed RHS
  int rhs_stages;     // tile: most x planes in the streamed RHS's ring
  int afx_planes;     // tile: x planes per block of the FP32 x factor
  int sm_reserved;    // SMs the structural update holds while the pressure solve runs
  int mixed_tc;       // mixed solve at 256 x 256: 1 = tensor-core predictor, 0 = FFT predictor
  int corr_bf16;      // mixed solve: the correction is stored in bfloat16 (FFT predictor path)
  float f_inv_h, f_inv_h2, f_nu;   // FP32 copies
};

// the per-step scalar in the precision of the kernel
template <class T>
__device__ __forceinline__ T pick(double d, float f) {
  if constexpr (sizeof(T) == 8) return (T)d;
  else return (T)f;
}

constexpr int ERR_AF_RANGE = 1;     // implicit diffusion number outside range
constexpr int ERR_NONFINITE = 2;    // non-finite CFL speed
constexpr int ERR_TIMEOUT = 4;      // a bounded device-side wait ran out
constexpr int ERR_IB_BIN = 8;       // a bar marker outside the tile it was binned to

__host__ __device__ inline size_t plane(const Consts& c) { return (size_t)c.ny * c.nz; }
__host__ __device__ inline size_t idx3(const Consts& c, int i, int j, int k) {
  return ((size_t)i * c.ny + j) * c.nz + k;
}

__device__ inline int wrap(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions (blockDim.x multiple of 32, <= 1024). Result valid on
// thread 0. `scratch` needs 32 doubles of shared memory.
__device__ inline double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}
__device__ inline double block_max(double v, double* scratch) {
  v = warp_max(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_max(v);
  return v;
}

// atomic max of a non-negative double through its ordered bit pattern
__device__ inline void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

}  // namespace ibm
