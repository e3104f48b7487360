// Host-side view of the device data of one solver state, and the kernel
// launchers each translation unit provides.
#pragma once

#include <vector>

#include "common.cuh"

namespace ibm {

template <class T>
struct Fields {
  T* u[2]; T* v[2]; T* w[2];  // velocity, double-buffered across the projection
  T* p;                       // pressure (nx * ny * nz)
  T* n[3];                    // nonlinear term N^{n-1}, overwritten with N^n
  T* d[3];                    // RHS, then the velocity increments
  T* e[3];                    // second buffer of the implicit line solves
  double* ipt;                // x-factor LU inverse pivots (2 x (nx + 2)), per step
  float* iptf;                // the same in FP32
  double* taps;               // periodic inverse taps along y (ny), z (nz), then free-space x taps
  float* tapsf;               // the same in FP32
  T* phi;                     // divergence -> transforms -> pressure correction
  T* ptab;                    // Poisson Thomas inverse pivots per distinct mode
  int* pconv;                 // per distinct mode: first plane from which its pivots equal the limit
  T* dout[3];                 // outflow-plane increments (ny * nz each)
  T* tw_y; T* tw_z;           // FFT twiddles exp(-2 pi i t / N), t < N/2 (re, im)
  double* partial;            // per-block partial maxima of the CFL speed
  double* qpart;              // per-block inflow/outflow flux partials
  double* mean00;             // line mean of the Poisson mode (0, 0)
  // prescribed inflow (null when disabled): 8 planes of ny * nz values:
  // pending u, v, w (next time level, written by the caller), current v, w
  // (ghosts of the explicit stage), increments u, v, w (x factor's first row)
  T* inflow;
  double* inflow_mean;        // mean of the pending u plane
  int n_partial;
  Params* prm;
};

struct Markers {
  int nm = 0;                 // flag vertices + bar markers
  int nf = 0;                 // flag vertices (markers 0 .. nf-1)
  int nb = 0;                 // bar markers
  double* Xb = nullptr;       // bar marker positions (3 per marker)
  double bar_dv = 0.0;        // volume carried by each bar marker
  double x_shift = 0.0;       // slab of an x decomposition: x of its first local plane (flag vertices
                              // are stored in global coordinates; bar markers are shifted once)
  double* coef = nullptr;     // 3 per marker: dV / h^3 * (U - U*)
  unsigned long long* acc = nullptr;   // deterministic mode: fixed-point sums, 3 fields
  size_t nfield = 0;                   // cells of one velocity field (accumulator stride)
  // Eulerian bar forcing: the velocity nodes whose cells the bars cut, u's
  // then v's then w's, with the solid fraction of each cell
  int nbm[3] = {0, 0, 0};
  int* bm_idx = nullptr;
  double* bm_alpha = nullptr;
  // bar markers binned by tiles of tx x ty x tz cells (Xb sorted by tile):
  // 5 ints per non-empty tile, its first cell (x, y, z) and bar range [b0, b1)
  int n_tiles = 0;
  int tx = 8, ty = 16, tz = 16;
  int* tile = nullptr;
  void* bar_w = nullptr;      // per bar marker: 18 kernel weights (field precision), set up once
  int* bar_o = nullptr;       // per bar marker: packed first box indices of its stencils
};

struct Flag {
  int ns = 0, nt = 0, nv = 0;
  double* X = nullptr;        // positions (3 per vertex)
  double* V = nullptr;        // velocities
  double* A = nullptr;        // accelerations (velocity Verlet)
  double* Ff = nullptr;       // fluid force on each vertex, -F_l dV_l
  double* inv_mass = nullptr; // 1/m for free vertices, 0 for the hinged edge
  double* dv = nullptr;       // marker volume of each vertex (area * h)
  int n_spring = 0;
  int* spring = nullptr;      // 2 vertex ids per spring
  double* l0 = nullptr;       // rest lengths
  double k_s = 0.0;
  int n_tri = 0;
  int* tri = nullptr;         // 3 vertex ids per triangle (both triangulations)
  int* tri_nb = nullptr;      // 3 per triangle: triangle across each hinge, or -1
  double* tri_k = nullptr;    // 3 per triangle: stiffness of that hinge
  double* tri_n = nullptr;    // 3 per triangle: unit normal (scratch)
  double* tri_inv = nullptr;  // 1 per triangle: 1 / |N| (scratch)
  double* slot = nullptr;     // 3 doubles per force slot: 3 per triangle, then 2 per spring
  int* csr_off = nullptr;     // nv + 1 offsets into csr_idx
  int* csr_idx = nullptr;     // slot ids contributing to each vertex
  int cluster = 1;            // CTAs cooperating in the structure kernel
};

// one case of a batched explicit stage: its constants, step parameters,
// fields of the current buffer parity, its block grid (x, y, z) and the index
// of its first block in the concatenated block list
template <class T>
struct RhsCase {
  Consts c;
  const Params* prm;
  const T *u, *v, *w, *p;
  T *n0, *n1, *n2, *d0, *d1, *d2;
  const T *vin, *win;
  int gx, gy, gz, first;
};

// one slab of the x decomposition of a case (slab.cu): owned cell planes
// [x_begin, x_end) of the global grid at local planes [gL, gL + n); gL, gR
// overlap planes on the sides with a neighbour; first_phys / last_phys: the
// slab holds the inflow / outflow end. Device tables: inverse pivots of the
// slab's rows per distinct mode (n x modes), six Green's-column values per
// mode, and a scratch of n x ny x nz values.
constexpr int SLAB_MAX_RANKS = 8;
constexpr int SLAB_LINE = 9;   // values per line in the all-gather of the pressure solve
struct SlabDev {
  int nranks = 1, rank = 0, x_begin = 0, x_end = 0, nx_global = 0;
  int n = 0, gL = 0, gR = 0, g = 0, first_phys = 1, last_phys = 1;
  double* tab = nullptr;
  double* green = nullptr;
  double* scr = nullptr;
};

// ---- fluid.cu
template <class T> void launch_begin_step(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_speed_check(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_af_tables(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_inflow(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_rhs(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> RhsCase<T> rhs_case(const Consts& c, const Fields<T>& f, int cur);
// the explicit stage of every case of `table` (device memory, ncases
// entries, `first` set) in one persistent launch of `blocks` blocks
template <class T> void launch_rhs_cases(const RhsCase<T>* table, int ncases, int total, int blocks, cudaStream_t s);
template <class T> void launch_outflow(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_af(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_af_x(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_af_y(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_af_z(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> bool launch_af_yz(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> bool launch_dht2d(const Consts& c, const Fields<T>& f, cudaStream_t s);
// FP32 2-D transform of every 256 x 256 plane from `in` to `out` (may alias); false for other shapes
bool launch_dht2d_on(const Consts& c, const Fields<float>& f, const float* in, float* out, cudaStream_t s);
bool dht2d_planes_fp32(const float* in, float* out, int nplanes, const float* tw, cudaStream_t s);
template <class T> void launch_mass(const Consts& c, const Fields<T>& f, int cur, cudaStream_t s);
template <class T> void launch_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s);
// phi = phi_a (f.phi when null) + phi_b (FP32) or + phi_b16 (bfloat16, FP32 fields only)
template <class T> void launch_project_only(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s,
                                            const T* phi_a = nullptr, const T* phi_b = nullptr,
                                            const void* phi_b16 = nullptr);
template <class T> void launch_mass_div(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s);
template <class T> void launch_project(const Consts& c, const Fields<T>& f, int cur, bool initial, cudaStream_t s,
                                       const T* phi_a = nullptr, const T* phi_b = nullptr,
                                       const void* phi_b16 = nullptr);
template <class T>
int partial_count(const Consts& c);
size_t poisson_table_size(const Consts& c);
size_t poisson_modes(const Consts& c);
// tensor-core (tcgen05) split-TF32 transform pass: out = (X H)^T per n x n
// plane (n = 32, 64, 128, 256), H the Hartley matrix given by its pre-split
// cos / sin image
bool tc_supported(int n);
size_t tc_h_image_bytes(int n);
void tc_pack_hartley(int n, unsigned char* img, cudaStream_t s);
// BF16 storage, 256 x 256 planes only (tc_gemm.cu)
size_t tc_bf16_image_bytes();
bool tc_bf16_available(const void* X, int planes);   // the tensor map of X can be encoded
void tc_pack_hartley_bf16(unsigned char* img, cudaStream_t s);
bool tc_rows_times_h_bf16(const void* X, const unsigned char* img, void* out, int planes, int* error,
                          cudaStream_t s, int sm_reserved);
bool tc_rows_times_h_t(const float* X, const unsigned char* himg, float* out, int planes, int n, int* error,
                       cudaStream_t s, bool single = false, int sm_reserved = 0);
void tc_gemm_set_attributes();
int outflow_blocks(const Consts& c);
void fluid_set_attributes();
template <class T> void launch_stats(const Consts& c, const Fields<T>& f, int cur, double* out, cudaStream_t s);

// ---- poisson.cu
template <class T> void launch_poisson(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_dht_y(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_dht_z(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_poisson_x(const Consts& c, const Fields<T>& f, cudaStream_t s);
template <class T> void launch_poisson_x_on(const Consts& c, const Fields<T>& f, T* buf, cudaStream_t s);
void launch_poisson_x_bf16(const Consts& c, const Fields<float>& f, void* buf, cudaStream_t s);
template <class T> void launch_poisson_table(const Consts& c, const Fields<T>& f, cudaStream_t s);
void poisson_set_attributes();

// ---- mixed.cu
// leaves phi = e[1] + e[2] (predictor + correction; the projection sums them)
void launch_poisson_mixed(const Consts& c, const Fields<float>& f, const float* Hy, const float* Hz,
                          const unsigned char* Hy_img, const unsigned char* Hz_img, const unsigned char* H16_img,
                          cudaStream_t s);
void mixed_set_attributes();
void launch_residual_mixed(const Consts& c, const Fields<float>& f, cudaStream_t s);
void hartley_matrix(int n, float* host);

// ---- ib.cu
template <class T> void launch_ib(const Consts& c, const Fields<T>& f, const Markers& m,
                                  const Flag& fl, int cur, cudaStream_t s);
void ib_set_attributes();
template <class T> void launch_ib_setup(const Consts& c, const Fields<T>& f, const Markers& m, cudaStream_t s);
// bin the bar markers (3 doubles each, sorted in place) into tiles; fills
// the tile table (5 ints per tile) and the tile shape of m
void ib_bin_bars(const Consts& c, std::vector<double>& Xb, std::vector<int>& tiles, Markers& m);

// ---- slab.cu
void slab_tables(const Consts& c, const SlabDev& sd, cudaStream_t s);
// local solves of the slab's rows (phi after the forward transforms); SLAB_LINE values per line to send
void slab_local_solve(const Consts& c, const SlabDev& sd, const double* phi, double* send, cudaStream_t s);
// reduced systems from every slab's line values (rank-major), corrected solution into phi
void slab_correct(const Consts& c, const SlabDev& sd, double* phi, const double* gathered, cudaStream_t s);
// owned flag forces (3 per vertex) and the two end fluxes; their sums back into the state
void slab_pack_force(const Consts& c, const SlabDev& sd, const Flag& fl, const double* qpart, int nqb,
                     double* send, cudaStream_t s);
void slab_unpack_force(const Consts& c, Params* prm, const Flag& fl, const double* recv, cudaStream_t s);

// ---- flag.cu
void launch_flag(Params* prm, const Flag& fl, bool force, cudaStream_t s);
void launch_flag_stats(const Flag& fl, double* out, cudaStream_t s);
int flag_max_cluster();

}  // namespace ibm
