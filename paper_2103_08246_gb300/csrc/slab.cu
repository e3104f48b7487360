// Decomposition of one case into slabs of whole y-z planes along x, one per
// GPU (the solver's 1-D domain decomposition, Sec. II.B). Each slab state
// holds its owned planes plus `g` overlap planes on every side that has a
// neighbour, and runs the ordinary kernels over that window; the parts of the
// step that couple the whole x extent are done here:
//
// * the pressure equation's tridiagonal solve along x per transverse mode
//   (Sec. II.B: transforms in y and z, a tridiagonal system along x), by the
//   partition method: every slab solves its own rows with the neighbours'
//   values removed (a cut row keeps the interior diagonal -2 + lam), the
//   first and last values of that solution and of the two Green's columns
//   T^-1 e_first, T^-1 e_last give a small system for the values next to
//   every cut (two unknowns per cut, solved redundantly by every slab after an
//   all-gather), and a second local solve with those values moved to the
//   right-hand side gives the exact solution; the singular mode (0, 0) keeps
//   the pinned first row of the whole line and its line mean comes from the
//   slabs' partial sums, so the gauge is the single-domain one;
// * the flag's fluid force: each vertex counts on the slab that owns its x
//   position (an all-reduce sums the slabs' masked force vectors), and every
//   slab advances the same structure;
// * the inflow and outflow fluxes of the mass fix, which only the first and
//   the last slab see.
//
// Everything else is local: the explicit terms, the y and z factors, the
// forcing and the projection are plane-local up to one or two planes, and the
// x factor of the implicit step forgets a wrong boundary value like rho^d
// (rho < 1 its decay factor) over d planes, so the overlap holds the exact
// values whenever it is wider than that decay length plus the kernel support.
// The overlap planes are refreshed from the neighbours after every step.
#include <cuda_runtime.h>

#include "solver.h"

namespace ibm {

namespace {

__device__ inline double slab_lambda(const Consts& c, int m) {
  const int qz_n = c.nz / 2 + 1;
  const int qy = m / qz_n, qz = m - qy * qz_n;
  const double sy = sin(M_PI * qy / c.ny), sz = sin(M_PI * qz / c.nz);
  return -4.0 * sy * sy - 4.0 * sz * sz;
}

__device__ inline int slab_mode(const Consts& c, int jk) {
  const int ky = jk / c.nz, kz = jk - ky * c.nz;
  const int qy = ky <= c.ny / 2 ? ky : c.ny - ky, qz = kz <= c.nz / 2 ? kz : c.nz - kz;
  return qy * (c.nz / 2 + 1) + qz;
}

// Per distinct mode m: the inverse LU pivots of the slab's rows (h^2 units:
// off-diagonals 1, diagonal -2 + lam, -1 + lam on a physical end row, 1 on the
// pinned first row of mode (0, 0)), and the first / last values and sums of
// the Green's columns g1 = T^-1 e_first and g2 = T^-1 e_last.
__global__ void k_slab_table(Consts c, SlabDev sd) {
  const int qz_n = c.nz / 2 + 1;
  const int PT = (c.ny / 2 + 1) * qz_n;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= PT) return;
  const double lam = slab_lambda(c, m);
  const bool pinned = (m == 0) && sd.first_phys;
  const int n = sd.n;
  double cp = 0.0;
  for (int i = 0; i < n; ++i) {
    double diag = -2.0 + lam;
    if ((i == 0 && sd.first_phys) || (i == n - 1 && sd.last_phys)) diag = -1.0 + lam;
    if (pinned && i == 0) diag = 1.0;
    const double lower = i == 0 ? 0.0 : 1.0;
    const double prev_cp = (pinned && i == 1) ? 0.0 : cp;
    const double inv = 1.0 / (diag - lower * prev_cp);
    sd.tab[(size_t)i * PT + m] = inv;
    cp = inv;
  }
  auto upper_cp = [&](int i) { return (pinned && i == 0) ? 0.0 : sd.tab[(size_t)i * PT + m]; };
  // g2: the forward sweep of e_last is zero up to the last row
  double x = sd.tab[(size_t)(n - 1) * PT + m];
  double g2l = x, s2 = x;
  for (int i = n - 2; i >= 0; --i) {
    x = -upper_cp(i) * x;
    s2 += x;
  }
  const double g2f = x;
  // g1: forward sweep of e_first into the scratch, then back substitution
  double y = 0.0;
  for (int i = 0; i < n; ++i) {
    const double rhs = i == 0 ? 1.0 : 0.0;
    y = (rhs - y) * sd.tab[(size_t)i * PT + m];
    sd.scr[(size_t)i * PT + m] = y;
  }
  x = y;
  double g1l = x, s1 = x;
  for (int i = n - 2; i >= 0; --i) {
    x = sd.scr[(size_t)i * PT + m] - upper_cp(i) * x;
    s1 += x;
  }
  const double g1f = x;
  double* gr = sd.green;
  gr[0 * (size_t)PT + m] = g1f;
  gr[1 * (size_t)PT + m] = g1l;
  gr[2 * (size_t)PT + m] = g2f;
  gr[3 * (size_t)PT + m] = g2l;
  gr[4 * (size_t)PT + m] = s1;
  gr[5 * (size_t)PT + m] = s2;
}

// Thomas solve of the slab's rows for line jk: rhs_i = scale * phi[gL + i]
// (0 on the pinned row) minus `left` on the first and `right` on the last row;
// the forward sweep goes to the scratch, back substitution calls out(i, x)
// from the last row down
template <class OUT>
__device__ inline void slab_thomas(const Consts& c, const SlabDev& sd, const double* phi, int jk, double scale,
                                   double left, double right, OUT out) {
  const int P = c.ny * c.nz, PT = (c.ny / 2 + 1) * (c.nz / 2 + 1);
  const int m = slab_mode(c, jk);
  const bool pinned = (jk == 0) && sd.first_phys;
  const int n = sd.n;
  double y = 0.0;
  for (int i = 0; i < n; ++i) {
    double rhs = (pinned && i == 0) ? 0.0 : phi[(size_t)(sd.gL + i) * P + jk] * scale;
    if (i == 0) rhs -= left;
    if (i == n - 1) rhs -= right;
    y = (rhs - y) * sd.tab[(size_t)i * PT + m];
    sd.scr[(size_t)i * P + jk] = y;
  }
  double x = y;
  out(n - 1, x);
  for (int i = n - 2; i >= 0; --i) {
    const double cp = (pinned && i == 0) ? 0.0 : sd.tab[(size_t)i * PT + m];
    x = sd.scr[(size_t)i * P + jk] - cp * x;
    out(i, x);
  }
}

// local solve of every line: 9 values per line for the all-gather
//   y_first, y_last, sum y, g1_first, g1_last, g2_first, g2_last, sum g1, sum g2
__global__ void __launch_bounds__(128) k_slab_local(Consts c, SlabDev sd, const double* __restrict__ phi,
                                                   double scale, double* __restrict__ send) {
  const int P = c.ny * c.nz, PT = (c.ny / 2 + 1) * (c.nz / 2 + 1);
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  double yf = 0.0, yl = 0.0, sy = 0.0;
  const int n = sd.n;
  slab_thomas(c, sd, phi, jk, scale, 0.0, 0.0, [&](int i, double x) {
    if (i == n - 1) yl = x;
    if (i == 0) yf = x;
    sy += x;
  });
  const int m = slab_mode(c, jk);
  double* o = send + (size_t)SLAB_LINE * jk;
  o[0] = yf;
  o[1] = yl;
  o[2] = sy;
  for (int q = 0; q < 6; ++q) o[3 + q] = sd.green[(size_t)q * PT + m];
}

// the values next to every cut from all slabs' line data (rank-major), then
// the slab's corrected solution (minus the line mean on mode (0, 0)); planes
// outside the owned rows are zeroed
__global__ void __launch_bounds__(128) k_slab_correct(Consts c, SlabDev sd, double* __restrict__ phi, double scale,
                                                     const double* __restrict__ gath, double inv_nx) {
  const int P = c.ny * c.nz;
  const int jk = blockIdx.x * blockDim.x + threadIdx.x;
  if (jk >= P) return;
  const int R = sd.nranks, M = 2 * (R - 1);
  // unknowns: L_k (last value of slab k, k <= R-2) at 2k, F_k (first value
  // of slab k, k >= 1) at 2k - 1; slab k's values are y_k - L_{k-1} g1_k - F_{k+1} g2_k
  double A[2 * (SLAB_MAX_RANKS - 1)][2 * (SLAB_MAX_RANKS - 1)];
  double b[2 * (SLAB_MAX_RANKS - 1)];
  for (int r = 0; r < M; ++r) {
    b[r] = 0.0;
    for (int q = 0; q < M; ++q) A[r][q] = 0.0;
  }
  auto line = [&](int k) { return gath + (size_t)k * SLAB_LINE * P + (size_t)SLAB_LINE * jk; };
  for (int k = 0; k < R; ++k) {
    const double* e = line(k);
    if (k >= 1) {   // F_k + g1f L_{k-1} + g2f F_{k+1} = y_first
      const int row = 2 * k - 1;
      A[row][row] = 1.0;
      A[row][2 * (k - 1)] += e[3];
      if (k <= R - 2) A[row][2 * k + 1] += e[5];
      b[row] = e[0];
    }
    if (k <= R - 2) {   // L_k + g1l L_{k-1} + g2l F_{k+1} = y_last
      const int row = 2 * k;
      A[row][row] = 1.0;
      if (k >= 1) A[row][2 * (k - 1)] += e[4];
      A[row][2 * k + 1] += e[6];
      b[row] = e[1];
    }
  }
  // Gaussian elimination with partial pivoting
  for (int col = 0; col < M; ++col) {
    int piv = col;
    for (int r = col + 1; r < M; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col) {
      for (int q = 0; q < M; ++q) {
        const double t = A[col][q];
        A[col][q] = A[piv][q];
        A[piv][q] = t;
      }
      const double t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
    const double inv = 1.0 / A[col][col];
    for (int r = col + 1; r < M; ++r) {
      const double f = A[r][col] * inv;
      if (f == 0.0) continue;
      for (int q = col; q < M; ++q) A[r][q] -= f * A[col][q];
      b[r] -= f * b[col];
    }
  }
  for (int r = M - 1; r >= 0; --r) {
    double acc = b[r];
    for (int q = r + 1; q < M; ++q) acc -= A[r][q] * b[q];
    b[r] = acc / A[r][r];
  }
  const int k = sd.rank;
  const double left = k >= 1 ? b[2 * (k - 1)] : 0.0;
  const double right = k <= R - 2 ? b[2 * k + 1] : 0.0;
  double mean = 0.0;
  if (jk == 0) {
    double tot = 0.0;
    for (int q = 0; q < R; ++q) {
      const double* e = line(q);
      tot += e[2];
      if (q >= 1) tot -= b[2 * (q - 1)] * e[7];
      if (q <= R - 2) tot -= b[2 * q + 1] * e[8];
    }
    mean = tot * inv_nx;
  }
  slab_thomas(c, sd, phi, jk, scale, left, right, [&](int i, double x) {
    phi[(size_t)(sd.gL + i) * P + jk] = x - mean;
  });
  for (int i = 0; i < sd.gL; ++i) phi[(size_t)i * P + jk] = 0.0;
  for (int i = sd.gL + sd.n; i < c.nx; ++i) phi[(size_t)i * P + jk] = 0.0;
}

// the flag's fluid force on the vertices this slab owns (x in [x_lo, x_hi);
// no bound on a physical end), zero elsewhere
__global__ void k_slab_pack_force(SlabDev sd, Flag fl, double x_lo, double x_hi, double* __restrict__ send) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= fl.nv) return;
  const double X = fl.X[3 * l];
  const bool own = (sd.first_phys || X >= x_lo) && (sd.last_phys || X < x_hi);
  for (int q = 0; q < 3; ++q) send[3 * l + q] = own ? fl.Ff[3 * l + q] : 0.0;
}

// the inflow flux (first slab) and outflow flux (last slab) as sums of the
// outflow kernel's block partials, in the order the single-domain mass fix sums them
__global__ void k_slab_pack_flux(SlabDev sd, const double* __restrict__ qpart, int nb, double* __restrict__ send) {
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
    send[0] = sd.first_phys ? qi : 0.0;
    send[1] = sd.last_phys ? qo : 0.0;
  }
}

// the summed forces and fluxes: force into the structure, mass-fix shift
// (Q_in - Q_out) / (Ly Lz) into the parameters
__global__ void k_slab_unpack_force(Consts c, Params* prm, Flag fl, const double* __restrict__ recv) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < 3 * fl.nv) fl.Ff[l] = recv[l];
  if (l == 0) {
    const double qi = recv[3 * fl.nv], qo = recv[3 * fl.nv + 1];
    const double h2 = c.h * c.h;
    prm->q_in = qi * h2;
    prm->q_out = qo * h2;
    prm->mass_shift = (qi - qo) * h2 / (c.ly * c.lz);
    prm->f_mass_shift = (float)prm->mass_shift;
  }
}

}  // namespace

void slab_tables(const Consts& c, const SlabDev& sd, cudaStream_t s) {
  const int PT = (c.ny / 2 + 1) * (c.nz / 2 + 1);
  k_slab_table<<<(PT + 127) / 128, 128, 0, s>>>(c, sd);
}

void slab_local_solve(const Consts& c, const SlabDev& sd, const double* phi, double* send, cudaStream_t s) {
  const int P = c.ny * c.nz;
  const double scale = c.h * c.h / ((double)c.ny * c.nz);
  k_slab_local<<<(P + 127) / 128, 128, 0, s>>>(c, sd, phi, scale, send);
}

void slab_correct(const Consts& c, const SlabDev& sd, double* phi, const double* gathered, cudaStream_t s) {
  const int P = c.ny * c.nz;
  const double scale = c.h * c.h / ((double)c.ny * c.nz);
  k_slab_correct<<<(P + 127) / 128, 128, 0, s>>>(c, sd, phi, scale, gathered, 1.0 / sd.nx_global);
}

void slab_pack_force(const Consts& c, const SlabDev& sd, const Flag& fl, const double* qpart, int nqb,
                     double* send, cudaStream_t s) {
  if (fl.nv) {
    const double x_lo = sd.x_begin * c.h, x_hi = sd.x_end * c.h;
    k_slab_pack_force<<<(fl.nv + 255) / 256, 256, 0, s>>>(sd, fl, x_lo, x_hi, send);
  }
  k_slab_pack_flux<<<1, 1024, 0, s>>>(sd, qpart, nqb, send + 3 * (size_t)fl.nv);
}

void slab_unpack_force(const Consts& c, Params* prm, const Flag& fl, const double* recv, cudaStream_t s) {
  const int n = 3 * fl.nv > 1 ? 3 * fl.nv : 1;
  k_slab_unpack_force<<<(n + 255) / 256, 256, 0, s>>>(c, prm, fl, recv);
}

}  // namespace ibm
