// C ABI of the solver (declared in include/ibm.h): argument checks, host-side
// geometry of the immersed bodies (Sec. II.A), device workspace layout, the
// initial projection, and one captured CUDA graph per velocity buffer parity
// for the time step of Sec. II.B.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/ibm.h"
#include "async_copy.cuh"
#include "solver.h"

using namespace ibm;

namespace {

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ------------------------------------------------------------------ geometry
struct FlagGeom {
  int ns = 0, nt = 0;
  std::vector<double> X, inv_mass, dv;
  std::vector<int> spring;
  std::vector<double> l0;
  std::vector<int> tri, tri_nb;       // 3 per triangle
  std::vector<double> tri_k;          // 3 per triangle
  int n_hinge = 0;
  std::vector<int> csr_off, csr_idx;
  double omega_max = 0.0;
};

// Flag lattice (Sec. II.A): sheet of flag_len x flag_span, leading edge at
// x = flag_x_le, centred in y and z, pitched by pitch0 about the z axis.
// Springs on lattice edges and both diagonals; bending hinges on every edge
// shared by two triangles of one of the two triangulations (cells split along
// either diagonal), stiffness beta |e|^2 / A on lattice edges and
// 2 beta A / |e|^2 on diagonals, each triangulation weighted 1/2.
FlagGeom build_flag(const ibm_bodies& b, const ibm_domain& d, double h) {
  FlagGeom g;
  const int ns = b.flag_ns, nt = b.flag_nt;
  g.ns = ns;
  g.nt = nt;
  const int nv = ns * nt;
  const double ds = b.flag_len / (ns - 1), dtt = b.flag_span / (nt - 1);
  const double yc = 0.5 * d.ly, zc = 0.5 * d.lz;
  auto vid = [nt](int a, int c) { return a * nt + c; };
  g.X.resize(3 * nv);
  for (int a = 0; a < ns; ++a)
    for (int c = 0; c < nt; ++c) {
      const int v = vid(a, c);
      g.X[3 * v] = b.flag_x_le + a * ds * std::cos(b.pitch0);
      g.X[3 * v + 1] = yc + a * ds * std::sin(b.pitch0);
      g.X[3 * v + 2] = zc - 0.5 * b.flag_span + c * dtt;
    }
  // lumped areas: a quarter of every adjacent cell
  std::vector<double> area(nv, 0.0);
  for (int a = 0; a + 1 < ns; ++a)
    for (int c = 0; c + 1 < nt; ++c) {
      const double q = 0.25 * ds * dtt;
      area[vid(a, c)] += q;
      area[vid(a + 1, c)] += q;
      area[vid(a, c + 1)] += q;
      area[vid(a + 1, c + 1)] += q;
    }
  g.inv_mass.resize(nv);
  g.dv.resize(nv);
  for (int v = 0; v < nv; ++v) {
    const bool pinned = v < nt;  // a = 0: the hinged leading edge
    g.inv_mass[v] = pinned ? 0.0 : 1.0 / (b.mass_ratio * area[v]);
    g.dv[v] = area[v] * h;
  }
  // springs
  auto add_spring = [&](int p, int q) {
    g.spring.push_back(p);
    g.spring.push_back(q);
    double s = 0.0;
    for (int e = 0; e < 3; ++e) {
      const double dd = g.X[3 * q + e] - g.X[3 * p + e];
      s += dd * dd;
    }
    g.l0.push_back(std::sqrt(s));
  };
  for (int a = 0; a < ns; ++a)
    for (int c = 0; c < nt; ++c) {
      if (a + 1 < ns) add_spring(vid(a, c), vid(a + 1, c));
      if (c + 1 < nt) add_spring(vid(a, c), vid(a, c + 1));
    }
  for (int a = 0; a + 1 < ns; ++a)
    for (int c = 0; c + 1 < nt; ++c) {
      add_spring(vid(a, c), vid(a + 1, c + 1));
      add_spring(vid(a + 1, c), vid(a, c + 1));
    }
  // two triangulations, triangles counter-clockwise in the (s, t) plane
  std::vector<std::array<int, 3>> tris;
  std::vector<int> kind;
  for (int split = 0; split < 2; ++split)
    for (int a = 0; a + 1 < ns; ++a)
      for (int c = 0; c + 1 < nt; ++c) {
        const int v00 = vid(a, c), v10 = vid(a + 1, c), v01 = vid(a, c + 1), v11 = vid(a + 1, c + 1);
        if (split == 0) {
          tris.push_back({v00, v10, v11});
          tris.push_back({v00, v11, v01});
        } else {
          tris.push_back({v00, v10, v01});
          tris.push_back({v10, v11, v01});
        }
        kind.push_back(split);
        kind.push_back(split);
      }
  std::map<std::tuple<int, int, int>, std::vector<int>> edges;
  for (int t = 0; t < (int)tris.size(); ++t)
    for (int e = 0; e < 3; ++e) {
      const int p = tris[t][e], q = tris[t][(e + 1) % 3];
      edges[std::make_tuple(kind[t], std::min(p, q), std::max(p, q))].push_back(t);
    }
  const int ntri = (int)tris.size();
  g.tri.resize(3 * ntri);
  for (int t = 0; t < ntri; ++t)
    for (int e = 0; e < 3; ++e) g.tri[3 * t + e] = tris[t][e];
  g.tri_nb.assign(3 * ntri, -1);
  g.tri_k.assign(3 * ntri, 0.0);
  std::vector<int> fill(ntri, 0);
  std::vector<std::array<int, 2>> hinge_tris;
  std::vector<double> hinge_k;
  const double cell = ds * dtt;
  for (auto& kv : edges) {
    if (kv.second.size() != 2) continue;
    const int ta = kv.second[0], tb = kv.second[1];
    const int p = std::get<1>(kv.first), q = std::get<2>(kv.first);
    const int ap = p / nt, cp = p % nt, aq = q / nt, cq = q % nt;
    const double es = (aq - ap) * ds, et = (cq - cp) * dtt;
    const double e2 = es * es + et * et;
    const bool diag = (aq != ap) && (cq != cp);
    const double k = 0.5 * (diag ? 2.0 * b.bending * cell / e2 : b.bending * e2 / cell);
    g.tri_nb[3 * ta + fill[ta]] = tb;
    g.tri_k[3 * ta + fill[ta]++] = k;
    g.tri_nb[3 * tb + fill[tb]] = ta;
    g.tri_k[3 * tb + fill[tb]++] = k;
    hinge_tris.push_back({ta, tb});
    hinge_k.push_back(k);
  }
  g.n_hinge = (int)hinge_k.size();
  // per-vertex slot lists (triangles: 3 slots, springs: 2 slots), fixed order
  const int nsp = (int)g.l0.size();
  std::vector<std::vector<int>> lists(nv);
  for (int t = 0; t < ntri; ++t)
    for (int e = 0; e < 3; ++e) lists[g.tri[3 * t + e]].push_back(3 * t + e);
  for (int q = 0; q < nsp; ++q) {
    lists[g.spring[2 * q]].push_back(3 * ntri + 2 * q);
    lists[g.spring[2 * q + 1]].push_back(3 * ntri + 2 * q + 1);
  }
  g.csr_off.assign(nv + 1, 0);
  for (int v = 0; v < nv; ++v) {
    g.csr_off[v + 1] = g.csr_off[v] + (int)lists[v].size();
    for (int sidx : lists[v]) g.csr_idx.push_back(sidx);
  }
  // Gershgorin bound of the stiffness / mass spectrum (linearised, flat):
  // (2 k_s n_springs(v) + 8 sum_hinges_at_v k_e / l_min^2) / m_v, free vertices
  std::vector<double> nspr(nv, 0.0), khs(nv, 0.0);
  for (int q = 0; q < nsp; ++q) {
    nspr[g.spring[2 * q]] += 1.0;
    nspr[g.spring[2 * q + 1]] += 1.0;
  }
  for (int q = 0; q < g.n_hinge; ++q) {
    int vs[6];
    for (int e = 0; e < 3; ++e) {
      vs[e] = tris[hinge_tris[q][0]][e];
      vs[3 + e] = tris[hinge_tris[q][1]][e];
    }
    std::sort(vs, vs + 6);
    const int* end = std::unique(vs, vs + 6);
    for (const int* p = vs; p != end; ++p) khs[*p] += hinge_k[q];
  }
  const double lmin = std::min(ds, dtt);
  double w2 = 0.0;
  for (int v = nt; v < nv; ++v) {
    const double m = b.mass_ratio * area[v];
    w2 = std::max(w2, (2.0 * b.stretch * nspr[v] + 8.0 * khs[v] / (lmin * lmin)) / m);
  }
  g.omega_max = std::sqrt(w2);
  return g;
}

// Bar-grid markers (Sec. II.A passive grid): rods along y centred at
// z = (r + 1/2) M and rods along z centred at y = (r + 1/2) M in the plane
// x = bar_x, each filled with n_w = ceil(d / h) + 1 points across both short
// sides and ceil(L / h) points along, at (m + 1/2) L / n. Points of rods along y
// inside a rod along z are dropped (crossings counted once). Each marker
// carries volume (union of the bars) / count.
void build_bars(const ibm_bodies& b, const ibm_domain& d, double h, std::vector<double>& X,
                double& dv) {
  const double dw = b.bar_width, M = b.bar_mesh;
  const int nry = (int)std::lround(d.ly / M), nrz = (int)std::lround(d.lz / M);
  const int nw = (int)std::ceil(dw / h - 1e-12) + 1;
  const int nay = (int)std::ceil(d.ly / h - 1e-12), naz = (int)std::ceil(d.lz / h - 1e-12);
  std::vector<double> across(nw);
  for (int q = 0; q < nw; ++q) across[q] = dw * ((double)q / (nw - 1) - 0.5);
  X.clear();
  for (int r = 0; r < nrz; ++r) {          // rods along y, centred in z
    const double z0 = (r + 0.5) * M;
    for (int qx = 0; qx < nw; ++qx)
      for (int qz = 0; qz < nw; ++qz)
        for (int m = 0; m < nay; ++m) {
          const double y = (m + 0.5) * d.ly / nay;
          bool inside = false;
          for (int s = 0; s < nry; ++s) {
            double dy = std::fabs(y - (s + 0.5) * M);
            dy = std::min(dy, d.ly - dy);
            if (dy <= 0.5 * dw + 1e-12) inside = true;
          }
          if (inside) continue;
          X.push_back(b.bar_x + across[qx]);
          X.push_back(y);
          X.push_back(z0 + across[qz]);
        }
  }
  for (int r = 0; r < nry; ++r) {          // rods along z, centred in y
    const double y0 = (r + 0.5) * M;
    for (int qx = 0; qx < nw; ++qx)
      for (int qy = 0; qy < nw; ++qy)
        for (int m = 0; m < naz; ++m) {
          X.push_back(b.bar_x + across[qx]);
          X.push_back(y0 + across[qy]);
          X.push_back((m + 0.5) * d.lz / naz);
        }
  }
  const double vol = dw * dw * (nry * d.lz + nrz * d.ly) - (double)nry * nrz * dw * dw * dw;
  const size_t n = X.size() / 3;
  dv = n ? vol / (double)n : 0.0;
}

// ------------------------------------------------------------------ workspace
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class P>
  P* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
    off += count * sizeof(P);
    return p;
  }
};

struct Layout {
  int nf = 0, nb = 0, nsp = 0, ntri = 0, nslot = 0, ncsr = 0;
  int nbm[3] = {0, 0, 0};   // Eulerian bar forcing: forced nodes per component
  int ntile = 0;            // tiles of the binned bar markers
};

// Eulerian forcing of the bar grid: for every velocity node whose cell
// [x - h/2, x + h/2]^3 the bars cut, its field index and the solid fraction
// alpha of the cell. The solid is the union of the rods (side d, in the slab
// |x - bar_x| <= d/2; along y centred at z = (r + 1/2) M, along z centred at
// y = (r + 1/2) M, periodic); with ox, oy, oz the cell's overlaps with the
// slab and with the rods across y and z,
// alpha h^3 = ox (h oz + oy h - oy oz).
struct BarMask {
  std::vector<int> idx;
  std::vector<double> alpha;
  int n[3] = {0, 0, 0};
  std::vector<int> tiles;   // bar markers: tile table of the binned markers
};

double cell_overlap(double c, double h, double lo, double hi) {
  return std::max(0.0, std::min(c + 0.5 * h, hi) - std::max(c - 0.5 * h, lo));
}

double rod_overlap(double c, double h, double d, double M, int nrods, double period) {
  double o = 0.0;
  for (int r = 0; r < nrods; ++r)
    for (int img = -1; img <= 1; ++img) {
      const double c0 = (r + 0.5) * M + img * period;
      o += cell_overlap(c, h, c0 - 0.5 * d, c0 + 0.5 * d);
    }
  return o;
}

void build_bar_mask(const ibm_bodies& b, const ibm_domain& dm, const ibm_grid& g, double h, BarMask& bm) {
  const double d = b.bar_width, M = b.bar_mesh;
  const int nry = (int)std::lround(dm.ly / M), nrz = (int)std::lround(dm.lz / M);
  bm.idx.clear();
  bm.alpha.clear();
  for (int comp = 0; comp < 3; ++comp) {
    const int ilo = comp == 0 ? 1 : 0, ihi = g.nx - 1;   // unknown planes of the component
    std::vector<double> oy(g.ny), oz(g.nz);
    for (int j = 0; j < g.ny; ++j) oy[j] = rod_overlap((j + (comp == 1 ? 0.0 : 0.5)) * h, h, d, M, nry, dm.ly);
    for (int k = 0; k < g.nz; ++k) oz[k] = rod_overlap((k + (comp == 2 ? 0.0 : 0.5)) * h, h, d, M, nrz, dm.lz);
    const size_t before = bm.idx.size();
    for (int i = ilo; i <= ihi; ++i) {
      const double x = (i + (comp == 0 ? 0.0 : 0.5)) * h;
      const double ox = cell_overlap(x, h, b.bar_x - 0.5 * d, b.bar_x + 0.5 * d);
      if (ox <= 0.0) continue;
      for (int j = 0; j < g.ny; ++j)
        for (int k = 0; k < g.nz; ++k) {
          const double a = ox * (h * oz[k] + oy[j] * h - oy[j] * oz[k]) / (h * h * h);
          if (a <= 0.0) continue;
          bm.idx.push_back((int)(((size_t)i * g.ny + j) * g.nz + k));
          bm.alpha.push_back(std::min(a, 1.0));
        }
    }
    bm.n[comp] = (int)(bm.idx.size() - before);
  }
}

}  // namespace

// ------------------------------------------------------------------ state
enum { GRAPH_HEAD = 0, GRAPH_MID = 1, GRAPH_TAIL = 2, GRAPH_KINDS = 3 };

struct ibm_state {
  int precision = IBM_FP64;
  bool deterministic = false;
  bool inflow = false;
  int bar_forcing = 0;   // 0: bar markers, 1: Eulerian volume-fraction forcing
  int* probes = nullptr;  // virtual probes: cell (i, j, k) index triples (own allocation)
  int nprobe = 0;
  Consts c{};
  ibm_grid grid{};
  ibm_domain dom{};
  ibm_bodies bodies{};
  double cfl = 0.3, cfl_limit = 2.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  int cur = 0;
  cudaGraphExec_t exec[GRAPH_KINDS][2] = {};
  cudaGraph_t graph[GRAPH_KINDS][2] = {};      // kept for ensembles
  Fields<double> fd{};
  Fields<float> ff{};
  Markers mk{};
  Flag fl{};
  Params* prm = nullptr;
  double* dstat = nullptr;    // 16 doubles of device scratch for diagnostics
  Params* hprm = nullptr;     // pinned copy
  double last_dt_fixed = -2.0;
  int kernels_per_step = 0;
  float* hy = nullptr;                    // Hartley matrices (mixed precision)
  float* hz = nullptr;
  unsigned char* hy_img = nullptr;        // pre-split tensor-core images of them (square planes)
  unsigned char* hz_img = nullptr;
  unsigned char* h16_img = nullptr;       // bfloat16 cos / sin image (256 x 256 planes, bfloat16 correction)
  cudaStream_t side = nullptr;            // structural update, overlapped in the graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t side2 = nullptr;           // implicit-factor tables, overlapped with the RHS
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  // slab of an x decomposition (ibm_create_slab): its geometry and solve
  // tables, the phases allowed next (bit mask), and whether the pending
  // projection is the initial one
  bool slab_on = false;
  SlabDev slab{};
  int slab_allowed = 0;
  bool slab_initial = false;
};

namespace {

int check_args(const ibm_grid* g, const ibm_domain* d, const ibm_bodies* b, const ibm_options* o) {
  if (!g || !d || !b) return IBM_EINVAL;
  if (g->nx < 4 || !is_pow2(g->ny) || !is_pow2(g->nz) || g->ny < 4 || g->nz < 4 || g->ny > 1024 ||
      g->nz > 1024 || g->nx > 65536)
    return IBM_EINVAL;
  if (!(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0)) return IBM_EINVAL;
  const double h = d->lx / g->nx;
  if (std::fabs(d->ly / g->ny - h) > 1e-9 * h || std::fabs(d->lz / g->nz - h) > 1e-9 * h)
    return IBM_EINVAL;
  if (b->bars_on) {
    if (!(b->bar_mesh > 0) || !(b->bar_width > 0) || b->bar_width >= b->bar_mesh) return IBM_EINVAL;
    const double ry = d->ly / b->bar_mesh, rz = d->lz / b->bar_mesh;
    if (std::fabs(ry - std::round(ry)) > 1e-9 || std::fabs(rz - std::round(rz)) > 1e-9) return IBM_EINVAL;
    if (b->bar_x - 0.5 * b->bar_width < 2 * h || b->bar_x + 0.5 * b->bar_width > d->lx - 2 * h)
      return IBM_EINVAL;
  }
  if (b->flag_on) {
    if (b->flag_ns < 2 || b->flag_nt < 2 || b->flag_ns * b->flag_nt > (1 << 20)) return IBM_EINVAL;
    if (!(b->flag_len > 0) || !(b->flag_span > 0) || !(b->mass_ratio > 0) || !(b->bending >= 0) ||
        !(b->stretch > 0))
      return IBM_EINVAL;
    if (b->flag_x_le < 2 * h || b->flag_x_le + b->flag_len > d->lx - 2 * h) return IBM_EINVAL;
  }
  if (o) {
    if (o->rhs_planes < 0 || o->rhs_planes > 256 || (o->rhs_planes > 0 && o->rhs_planes < 2) ||
        o->afx_planes < 0 || o->afx_planes > 256 || (o->afx_planes > 0 && o->afx_planes < 8) ||
        o->rhs_stages < 0 || o->rhs_stages > 8 || (o->rhs_stages > 0 && o->rhs_stages < 4))
      return IBM_EINVAL;
    if (o->precision != IBM_FP64 && o->precision != IBM_FP32 && o->precision != IBM_MIXED)
      return IBM_EINVAL;
    if (o->cfl < 0 || o->cfl_limit < 0) return IBM_EINVAL;
    if (o->bar_forcing != 0 && o->bar_forcing != 1) return IBM_EINVAL;
    if (o->mixed_tc_predictor != 0 && o->mixed_tc_predictor != 1) return IBM_EINVAL;
  }
  return IBM_OK;
}

template <class T>
size_t carve(ibm_state* s, void* base, const Layout& L, Fields<T>& f) {
  Carver cv(base);
  const Consts& c = s->c;
  const size_t NF = (size_t)(c.nx + 1) * c.ny * c.nz, NP = (size_t)c.nx * c.ny * c.nz;
  const size_t P = (size_t)c.ny * c.nz;
  for (int b = 0; b < 2; ++b) {
    f.u[b] = cv.take<T>(NF);
    f.v[b] = cv.take<T>(NF);
    f.w[b] = cv.take<T>(NF);
  }
  for (int q = 0; q < 3; ++q) f.n[q] = cv.take<T>(NF);
  for (int q = 0; q < 3; ++q) f.d[q] = cv.take<T>(NF);
  for (int q = 0; q < 3; ++q) f.e[q] = cv.take<T>(NF);
  f.ipt = cv.take<double>(2 * (size_t)(c.nx + 2));
  f.iptf = cv.take<float>(2 * (size_t)(c.nx + 2));
  f.taps = cv.take<double>((size_t)c.ny + c.nz + 32);
  f.tapsf = cv.take<float>((size_t)c.ny + c.nz + 32);
  f.p = cv.take<T>(NP);
  f.phi = cv.take<T>(NP);
  f.ptab = cv.take<T>(poisson_table_size(c));
  f.pconv = cv.take<int>(poisson_modes(c));
  for (int q = 0; q < 3; ++q) f.dout[q] = cv.take<T>(P);
  f.tw_y = cv.take<T>(c.ny);
  f.tw_z = cv.take<T>(c.nz);
  f.n_partial = partial_count<T>(c);
  f.partial = cv.take<double>(f.n_partial);
  f.qpart = cv.take<double>(2 * (size_t)outflow_blocks(c));
  f.mean00 = cv.take<double>(1);
  f.inflow = s->inflow ? cv.take<T>(8 * P) : nullptr;
  f.inflow_mean = s->inflow ? cv.take<double>(1) : nullptr;
  f.prm = cv.take<Params>(1);
  s->dstat = cv.take<double>(16);
  Markers& m = s->mk;
  m.nf = L.nf;
  m.nb = L.nb;
  m.nm = L.nf + L.nb;
  m.Xb = cv.take<double>(3 * (size_t)L.nb);
  m.coef = cv.take<double>(3 * (size_t)m.nm);
  m.nfield = NF;
  m.acc = s->deterministic ? cv.take<unsigned long long>(3 * NF) : nullptr;
  for (int q = 0; q < 3; ++q) m.nbm[q] = L.nbm[q];
  m.bm_idx = cv.take<int>((size_t)L.nbm[0] + L.nbm[1] + L.nbm[2]);
  m.bm_alpha = cv.take<double>((size_t)L.nbm[0] + L.nbm[1] + L.nbm[2]);
  m.n_tiles = L.ntile;
  m.tile = cv.take<int>(5 * (size_t)L.ntile);
  m.bar_w = L.ntile ? (void*)cv.take<T>(18 * (size_t)L.nb) : nullptr;
  m.bar_o = L.ntile ? cv.take<int>((size_t)L.nb) : nullptr;
  Flag& fl = s->fl;
  fl.nv = L.nf;
  fl.X = cv.take<double>(3 * (size_t)L.nf);
  fl.V = cv.take<double>(3 * (size_t)L.nf);
  fl.A = cv.take<double>(3 * (size_t)L.nf);
  fl.Ff = cv.take<double>(3 * (size_t)L.nf);
  fl.inv_mass = cv.take<double>(L.nf);
  fl.dv = cv.take<double>(L.nf);
  fl.n_spring = L.nsp;
  fl.spring = cv.take<int>(2 * (size_t)L.nsp);
  fl.l0 = cv.take<double>(L.nsp);
  fl.n_tri = L.ntri;
  fl.tri = cv.take<int>(3 * (size_t)L.ntri);
  fl.tri_nb = cv.take<int>(3 * (size_t)L.ntri);
  fl.tri_k = cv.take<double>(3 * (size_t)L.ntri);
  fl.tri_n = cv.take<double>(3 * (size_t)L.ntri);
  fl.tri_inv = cv.take<double>(L.ntri);
  fl.slot = cv.take<double>(3 * (size_t)L.nslot);
  fl.csr_off = cv.take<int>(L.nf + 1);
  fl.csr_idx = cv.take<int>(L.ncsr);
  s->prm = f.prm;
  if (s->precision == IBM_MIXED) {
    s->hy = cv.take<float>((size_t)c.ny * c.ny);
    s->hz = cv.take<float>((size_t)c.nz * c.nz);
    if (c.ny == c.nz && tc_supported(c.ny)) {
      s->hy_img = cv.take<unsigned char>(tc_h_image_bytes(c.ny));
      s->hz_img = cv.take<unsigned char>(tc_h_image_bytes(c.nz));
      if (c.ny == 256) s->h16_img = cv.take<unsigned char>(tc_bf16_image_bytes());
    }
  }
  return cv.off + 256;
}

#define CK(x)                          \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) {           \
      cudaGetLastError();              \
      return IBM_ECUDA;                \
    }                                  \
  } while (0)

template <class T>
Fields<T>& fields(ibm_state* s);
template <>
Fields<double>& fields<double>(ibm_state* s) { return s->fd; }
template <>
Fields<float>& fields<float>(ibm_state* s) { return s->ff; }

// FP64 host values <-> FP32 device field, converted on the device: the
// doubles travel through a device staging buffer in chunks
__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    b[q] = (double)a[q];
}

int upload_f32_staged(cudaStream_t st, float* dst, const double* src, size_t n, double* stage,
                      size_t cap) {
  for (size_t o = 0; o < n; o += cap) {
    const size_t m = std::min(cap, n - o);
    CK(cudaMemcpyAsync(stage, src + o, m * sizeof(double), cudaMemcpyHostToDevice, st));
    k_f64_to_f32<<<1024, 256, 0, st>>>(stage, dst + o, m);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

int download_f32_staged(cudaStream_t st, double* dst, const float* src, size_t n, double* stage,
                        size_t cap) {
  for (size_t o = 0; o < n; o += cap) {
    const size_t m = std::min(cap, n - o);
    k_f32_to_f64<<<1024, 256, 0, st>>>(src + o, stage, m);
    CK(cudaMemcpyAsync(dst + o, stage, m * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

template <class T>
int upload_field(cudaStream_t st, T* dst, const double* src, size_t n) {
  if (std::is_same<T, double>::value) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::vector<T> tmp(n);
    for (size_t i = 0; i < n; ++i) tmp[i] = (T)src[i];
    CK(cudaMemcpyAsync(dst, tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  return IBM_OK;
}

template <class T>
int download_field(cudaStream_t st, double* dst, const T* src, size_t n) {
  if (std::is_same<T, double>::value) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::vector<T> tmp(n);
    CK(cudaMemcpyAsync(tmp.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n; ++i) dst[i] = (double)tmp[i];
  }
  return IBM_OK;
}

template <class T>
void solve_poisson(ibm_state* s, cudaStream_t st) {
  Fields<T>& f = fields<T>(s);
  if constexpr (std::is_same<T, float>::value) {
    if (s->precision == IBM_MIXED) {
      launch_poisson_mixed(s->c, f, s->hy, s->hz, s->hy_img, s->hz_img, s->h16_img, st);
      return;
    }
  }
  launch_poisson(s->c, f, st);
}

// projection after solve_poisson: the mixed solve leaves phi as predictor
// (e[1]) plus correction (e[2]), which the projection sums as it reads them
template <class T>
void project_after_solve(ibm_state* s, int cur, bool initial, cudaStream_t st) {
  Fields<T>& f = fields<T>(s);
  if (std::is_same<T, float>::value && s->precision == IBM_MIXED && s->c.corr_bf16)
    launch_project(s->c, f, cur, initial, st, (const T*)f.e[1], (const T*)nullptr, (const void*)f.e[2]);
  else if (std::is_same<T, float>::value && s->precision == IBM_MIXED)
    launch_project(s->c, f, cur, initial, st, (const T*)f.e[1], (const T*)f.e[2]);
  else
    launch_project(s->c, f, cur, initial, st);
}

// A time step is split at the immersed-boundary forcing into a head (dt, RHS,
// implicit factors) and a tail (forcing, structure, pressure, projection).
// The structural update needs only the forcing's result and is needed only
// by the next step's forcing, so it runs on a side stream from the forcing of
// one step to the end of the next step's head. ibm_step(n) therefore replays
//   head(n0), mid x (n - 1), tail,   mid = tail of one step + head of the next,
// three captured graphs per velocity buffer parity; every replay ends with
// all its work (the structural update included) joined.
template <class T>
void record_head(ibm_state* s, int cur) {
  Fields<T>& f = fields<T>(s);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  launch_begin_step(c, f, st);
  // the implicit factors' tables for this step's r, concurrent with the RHS
  cudaEventRecord(s->ev_fork2, st);
  cudaStreamWaitEvent(s->side2, s->ev_fork2, 0);
  launch_af_tables(c, f, s->side2);
  cudaEventRecord(s->ev_join2, s->side2);
  launch_rhs(c, f, cur, st);
  launch_inflow(c, f, cur, st);   // new inflow time level (prescribed inflow only)
  launch_outflow(c, f, cur, st);
  cudaStreamWaitEvent(st, s->ev_join2, 0);
  launch_af(c, f, cur, st);
}

// forcing, structural update forked; returns whether a join is owed
template <class T>
bool record_tail_body(ibm_state* s, int cur) {
  Fields<T>& f = fields<T>(s);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  launch_ib(c, f, s->mk, s->fl, cur, st);
  const bool flag = s->fl.nv > 0;
  if (flag) {
    cudaEventRecord(s->ev_fork, st);
    cudaStreamWaitEvent(s->side, s->ev_fork, 0);
    launch_flag(f.prm, s->fl, false, s->side);
    cudaEventRecord(s->ev_join, s->side);
  }
  launch_mass_div(c, f, cur, false, st);
  solve_poisson<T>(s, st);
  project_after_solve<T>(s, cur, false, st);
  return flag;
}

template <class T>
void record_graph(ibm_state* s, int kind, int cur) {
  if (kind == GRAPH_HEAD) {
    record_head<T>(s, cur);
    return;
  }
  const bool join = record_tail_body<T>(s, cur);
  if (kind == GRAPH_MID) record_head<T>(s, cur ^ 1);
  if (kind == GRAPH_TAIL) launch_speed_check(s->c, fields<T>(s), s->stream);
  if (join) cudaStreamWaitEvent(s->stream, s->ev_join, 0);
}

template <class T>
int init_state(ibm_state* s, const ibm_options* o, const FlagGeom& fg,
               const std::vector<double>& Xb, double bar_dv, const BarMask& bm) {
  Fields<T>& f = fields<T>(s);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  const size_t NF = (size_t)(c.nx + 1) * c.ny * c.nz, NP = (size_t)c.nx * c.ny * c.nz;
  CK(cudaMemsetAsync(s->ws, 0, s->ws_bytes, st));
  // velocity: u = U + init_u, v = init_v, w = init_w
  {
    std::vector<double> buf(NF);
    for (int comp = 0; comp < 3; ++comp) {
      const double* src = o ? (comp == 0 ? o->init_u : comp == 1 ? o->init_v : o->init_w) : nullptr;
      for (size_t e = 0; e < NF; ++e) buf[e] = (comp == 0 ? c.u_in : 0.0) + (src ? src[e] : 0.0);
      T* dst = comp == 0 ? f.u[0] : comp == 1 ? f.v[0] : f.w[0];
      int rc = upload_field<T>(st, dst, buf.data(), NF);
      if (rc) return rc;
    }
  }
  // prescribed inflow: pending u = U, everything else zero (uniform (U, 0, 0))
  if (f.inflow) {
    std::vector<double> ones((size_t)c.ny * c.nz, c.u_in);
    int rc = upload_field<T>(st, f.inflow, ones.data(), ones.size());
    if (rc) return rc;
  }
  // twiddles exp(-2 pi i t / N)
  for (int dir = 0; dir < 2; ++dir) {
    const int n = dir == 0 ? c.ny : c.nz;
    std::vector<double> tw(n);
    for (int t = 0; t < n / 2; ++t) {
      tw[2 * t] = std::cos(2.0 * M_PI * t / n);
      tw[2 * t + 1] = -std::sin(2.0 * M_PI * t / n);
    }
    int rc = upload_field<T>(st, dir == 0 ? f.tw_y : f.tw_z, tw.data(), n);
    if (rc) return rc;
  }
  // markers and flag
  Markers& m = s->mk;
  m.bar_dv = bar_dv;
  if (m.nb) CK(cudaMemcpyAsync(m.Xb, Xb.data(), Xb.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (!bm.tiles.empty())
    CK(cudaMemcpyAsync(m.tile, bm.tiles.data(), bm.tiles.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!bm.idx.empty()) {
    CK(cudaMemcpyAsync(m.bm_idx, bm.idx.data(), bm.idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(m.bm_alpha, bm.alpha.data(), bm.alpha.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  Flag& fl = s->fl;
  if (fl.nv) {
    fl.ns = fg.ns;
    fl.nt = fg.nt;
    fl.k_s = s->bodies.stretch;
    auto up = [&](void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    CK(up(fl.X, fg.X.data(), fg.X.size() * sizeof(double)));
    CK(up(fl.inv_mass, fg.inv_mass.data(), fg.inv_mass.size() * sizeof(double)));
    CK(up(fl.dv, fg.dv.data(), fg.dv.size() * sizeof(double)));
    CK(up(fl.spring, fg.spring.data(), fg.spring.size() * sizeof(int)));
    CK(up(fl.l0, fg.l0.data(), fg.l0.size() * sizeof(double)));
    CK(up(fl.tri, fg.tri.data(), fg.tri.size() * sizeof(int)));
    CK(up(fl.tri_nb, fg.tri_nb.data(), fg.tri_nb.size() * sizeof(int)));
    CK(up(fl.tri_k, fg.tri_k.data(), fg.tri_k.size() * sizeof(double)));
    CK(up(fl.csr_off, fg.csr_off.data(), fg.csr_off.size() * sizeof(int)));
    CK(up(fl.csr_idx, fg.csr_idx.data(), fg.csr_idx.size() * sizeof(int)));
    // enough CTAs for the hinge work, within the cluster limit
    const int want = std::min((fl.n_tri + fl.n_spring + 1023) / 1024, flag_max_cluster());
    fl.cluster = 1;
    while (2 * fl.cluster <= want) fl.cluster *= 2;
    // the structural update runs beside the pressure solve: persistent
    // kernels there leave its SMs free instead of queueing behind it
    s->c.sm_reserved = fl.cluster;
  }
  // parameters
  Params p{};
  p.first = 1;
  p.dt_fixed = -1.0;
  p.cfl = s->cfl;
  CK(cudaMemcpyAsync(f.prm, &p, sizeof(Params), cudaMemcpyHostToDevice, st));
  ib_set_attributes();
  launch_ib_setup<T>(c, f, m, st);   // the bar markers' weights and box indices, once
  CK(cudaGetLastError());
  poisson_set_attributes();
  fluid_set_attributes();
  mixed_set_attributes();
  if (s->precision == IBM_MIXED) {
    std::vector<float> H((size_t)std::max(c.ny, c.nz) * std::max(c.ny, c.nz));
    hartley_matrix(c.ny, H.data());
    CK(cudaMemcpyAsync(s->hy, H.data(), (size_t)c.ny * c.ny * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    hartley_matrix(c.nz, H.data());
    CK(cudaMemcpyAsync(s->hz, H.data(), (size_t)c.nz * c.nz * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (s->hy_img) {
      tc_pack_hartley(c.ny, s->hy_img, st);
      tc_pack_hartley(c.nz, s->hz_img, st);
      if (s->h16_img) tc_pack_hartley_bf16(s->h16_img, st);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(st));
    }
    s->c.corr_bf16 = (s->h16_img && !s->c.mixed_tc && tc_bf16_available(fields<float>(s).e[2], c.nx)) ? 1 : 0;
  }
  launch_poisson_table(c, f, st);
  if (s->slab_on) {   // projected by the phase sequence; no captured step
    s->cur = 0;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    // the structural update runs beside the pressure phases
    CK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    return IBM_OK;
  }
  // initial projection of u0 (dt absorbed in phi), velocity only
  s->cur = 0;
  launch_mass_div(c, f, 0, true, st);
  solve_poisson<T>(s, st);
  project_after_solve<T>(s, 0, true, st);
  s->cur = 1;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  (void)NP;
  CK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&s->side2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->ev_fork2, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_join2, cudaEventDisableTiming));
  // capture head, mid and tail per buffer parity
  for (int kind = 0; kind < GRAPH_KINDS; ++kind)
    for (int par = 0; par < 2; ++par) {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      record_graph<T>(s, kind, par);
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return IBM_ECUDA;
      }
      if (kind == GRAPH_MID) {
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        s->kernels_per_step = (int)nodes;   // a steady-state step: tail + next head
      }
      e = cudaGraphInstantiate(&s->exec[kind][par], g, 0);
      s->graph[kind][par] = g;
      if (e != cudaSuccess) {
        cudaGetLastError();
        return IBM_ECUDA;
      }
    }
  return IBM_OK;
}

// the window of a slab: its first cell plane in the global grid and its planes
int slab_window(const ibm_slab& sl, int* x0, int* nxw) {
  const int gl = sl.rank > 0 ? sl.ghosts : 0, gr = sl.rank < sl.nranks - 1 ? sl.ghosts : 0;
  *x0 = sl.x_begin - gl;
  *nxw = sl.x_end - sl.x_begin + gl + gr;
  return gl;
}

int check_slab(const ibm_grid* g, const ibm_options* o, const ibm_slab* sl) {
  if (!sl || !g) return IBM_EINVAL;
  if (sl->nranks < 1 || sl->nranks > IBM_SLAB_MAX_RANKS || sl->rank < 0 || sl->rank >= sl->nranks)
    return IBM_EINVAL;
  if (sl->x_begin < 0 || sl->x_end <= sl->x_begin || sl->x_end > g->nx) return IBM_EINVAL;
  if ((sl->rank == 0) != (sl->x_begin == 0) || (sl->rank == sl->nranks - 1) != (sl->x_end == g->nx))
    return IBM_EINVAL;
  if (sl->nranks > 1 && (sl->ghosts < 1 || sl->x_end - sl->x_begin < sl->ghosts + 1)) return IBM_EINVAL;
  if (sl->ghosts < 0) return IBM_EINVAL;
  int x0, nxw;
  slab_window(*sl, &x0, &nxw);
  if (x0 < 0 || x0 + nxw > g->nx || nxw < 4) return IBM_EINVAL;
  if (o && (o->precision != IBM_FP64 || o->inflow || o->bar_forcing != 0)) return IBM_EINVAL;
  return IBM_OK;
}

int prepare(const ibm_grid* g, const ibm_domain* d, const ibm_bodies* b, const ibm_options* o,
            ibm_state* s, FlagGeom& fg, std::vector<double>& Xb, double& bar_dv, Layout& L, BarMask& bm,
            const ibm_slab* sl = nullptr) {
  int rc = check_args(g, d, b, o);
  if (rc) return rc;
  if (sl && (rc = check_slab(g, o, sl))) return rc;
  s->grid = *g;
  s->dom = *d;
  s->bodies = *b;
  s->precision = o ? o->precision : IBM_FP64;
  s->deterministic = o && o->deterministic;
  s->inflow = o && o->inflow;
  s->bar_forcing = o ? o->bar_forcing : 0;
  s->cfl = (o && o->cfl > 0) ? o->cfl : 0.3;
  s->cfl_limit = (o && o->cfl_limit > 0) ? o->cfl_limit : 2.0;
  Consts& c = s->c;
  c.nx = g->nx;
  c.ny = g->ny;
  c.nz = g->nz;
  c.h = d->lx / g->nx;
  c.inv_h = 1.0 / c.h;
  c.lx = d->lx;
  c.ly = d->ly;
  c.lz = d->lz;
  c.u_in = 1.0;
  c.f_inv_h = (float)c.inv_h;
  c.f_inv_h2 = (float)(c.inv_h * c.inv_h);
  c.rhs_planes = (o && o->rhs_planes > 0) ? o->rhs_planes : 16;
  c.rhs_stages = (o && o->rhs_stages > 0) ? o->rhs_stages : 8;
  c.afx_planes = (o && o->afx_planes > 0) ? o->afx_planes : 64;
  c.mixed_tc = o ? o->mixed_tc_predictor : 0;
  bar_dv = 0.0;
  if (b->flag_on) fg = build_flag(*b, *d, c.h);
  if (b->bars_on && s->bar_forcing == 1) build_bar_mask(*b, *d, *g, c.h, bm);
  else if (b->bars_on) build_bars(*b, *d, c.h, Xb, bar_dv);
  if (sl) {
    // the window: the global grid's bodies (flag in global coordinates,
    // shifted by the forcing kernels), bar markers within three cells of the
    // window shifted to window coordinates; the marker volume stays the
    // global grid's
    int x0, nxw;
    slab_window(*sl, &x0, &nxw);
    const double xs = x0 * c.h;
    std::vector<double> keep;
    for (size_t q = 0; q + 2 < Xb.size(); q += 3) {
      const long long cx = (long long)std::floor(Xb[q] * c.inv_h);
      if (cx < x0 - 3 || cx > x0 + nxw + 2) continue;
      keep.push_back(Xb[q] - xs);
      keep.push_back(Xb[q + 1]);
      keep.push_back(Xb[q + 2]);
    }
    Xb.swap(keep);
    c.nx = nxw;
    c.lx = nxw * c.h;
    s->grid.nx = nxw;
    s->dom.lx = c.lx;
    s->mk.x_shift = xs;
  }
  ib_bin_bars(c, Xb, bm.tiles, s->mk);
  L.ntile = s->mk.n_tiles;
  for (int q = 0; q < 3; ++q) L.nbm[q] = bm.n[q];
  c.omega_max = fg.omega_max;
  L.nf = b->flag_on ? b->flag_ns * b->flag_nt : 0;
  L.nb = (int)(Xb.size() / 3);
  L.nsp = (int)fg.l0.size();
  L.ntri = (int)(fg.tri.size() / 3);
  L.nslot = 2 * L.nsp + 3 * L.ntri;
  L.ncsr = (int)fg.csr_idx.size();
  return IBM_OK;
}

template <class T>
int step_impl(ibm_state* s, double dt, int nsteps) {
  Fields<T>& f = fields<T>(s);
  cudaStream_t st = s->stream;
  const double mode = dt > 0 ? dt : -1.0;
  if (mode != s->last_dt_fixed) {
    // dt_fixed and cfl are adjacent members of Params
    double two[2] = {mode, s->cfl};
    CK(cudaMemcpyAsync(&f.prm->dt_fixed, two, sizeof(two), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    s->last_dt_fixed = mode;
  }
  if (nsteps > 0) {
    CK(cudaGraphLaunch(s->exec[GRAPH_HEAD][s->cur], st));
    for (int n = 1; n < nsteps; ++n) {
      CK(cudaGraphLaunch(s->exec[GRAPH_MID][s->cur], st));
      s->cur ^= 1;
    }
    CK(cudaGraphLaunch(s->exec[GRAPH_TAIL][s->cur], st));
    s->cur ^= 1;
  }
  CK(cudaMemcpyAsync(s->hprm, f.prm, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const Params& p = *s->hprm;
  if (p.error & ERR_TIMEOUT) return IBM_ETIMEOUT;
  if (p.error & ERR_AF_RANGE) return IBM_EINVAL;
  if (p.error) return IBM_EDIVERGED;
  if (nsteps > 0 && p.dt * p.speed_max / s->c.h > s->cfl_limit) return IBM_EDIVERGED;
  return IBM_OK;
}

}  // namespace

namespace {
template <class T>
void launch_stage(ibm_state* s, int stage) {
  Fields<T>& f = fields<T>(s);
  const Consts& c = s->c;
  cudaStream_t st = s->stream;
  const int cur = s->cur;
  switch (stage) {
    case IBM_STAGE_RHS: launch_rhs(c, f, cur, st); break;
    case IBM_STAGE_OUTFLOW: launch_outflow(c, f, cur, st); break;
    case IBM_STAGE_AF_X: launch_af_x(c, f, cur, st); break;
    case IBM_STAGE_AF_Y: launch_af_y(c, f, cur, st); break;
    case IBM_STAGE_AF_Z: launch_af_z(c, f, cur, st); break;
    case IBM_STAGE_IB: launch_ib(c, f, s->mk, s->fl, cur, st); break;
    case IBM_STAGE_FLAG: launch_flag(f.prm, s->fl, true, st); break;
    case IBM_STAGE_MASS_DIV: launch_mass_div(c, f, cur, false, st); break;
    case IBM_STAGE_DHT_Y: launch_dht_y(c, f, st); break;
    case IBM_STAGE_DHT_Z: launch_dht_z(c, f, st); break;
    case IBM_STAGE_POISSON_X: launch_poisson_x(c, f, st); break;
    case IBM_STAGE_PROJECT:
      // as the step runs it: the mixed solve's two parts summed as they are read
      if (std::is_same<T, float>::value && s->precision == IBM_MIXED && c.corr_bf16)
        launch_project_only(c, f, cur, false, st, (const T*)f.e[1], (const T*)nullptr, (const void*)f.e[2]);
      else if (std::is_same<T, float>::value && s->precision == IBM_MIXED)
        launch_project_only(c, f, cur, false, st, (const T*)f.e[1], (const T*)f.e[2]);
      else
        launch_project_only(c, f, cur, false, st);
      break;
    case IBM_STAGE_POISSON: solve_poisson<T>(s, st); break;
    case IBM_STAGE_AF_YZ: (void)launch_af_yz(c, f, cur, st); break;
    case IBM_STAGE_DHT_2D: (void)launch_dht2d(c, f, st); break;
    case IBM_STAGE_TC_PASS:
      if constexpr (std::is_same<T, float>::value)
        if (s->precision == IBM_MIXED && s->hz_img)
          (void)tc_rows_times_h_t(f.phi, s->hz_img, f.e[0], c.nx, c.nz, &f.prm->error, st);
      break;
    case IBM_STAGE_TC_PASS1:
      if constexpr (std::is_same<T, float>::value)
        if (s->precision == IBM_MIXED && s->hz_img && c.nz == 256)
          (void)tc_rows_times_h_t(f.phi, s->hz_img, f.e[0], c.nx, c.nz, &f.prm->error, st, true);
      break;
    case IBM_STAGE_RESIDUAL:
      if constexpr (std::is_same<T, float>::value)
        if (s->precision == IBM_MIXED) launch_residual_mixed(c, f, st);
      break;
    case IBM_STAGE_TC_BF16:
      if constexpr (std::is_same<T, float>::value)
        if (s->precision == IBM_MIXED && c.corr_bf16)
          (void)tc_rows_times_h_bf16(f.e[2], s->h16_img, f.e[0], c.nx, &f.prm->error, st, c.sm_reserved);
      break;
    case IBM_STAGE_POISSON_X16:
      if constexpr (std::is_same<T, float>::value)
        if (s->precision == IBM_MIXED && c.corr_bf16) launch_poisson_x_bf16(c, f, f.e[2], st);
      break;
    default: break;
  }
}

}  // namespace

// ------------------------------------------------------------------ C ABI
namespace {

// cell-centred velocity at the probes: u from faces i, i + 1, v from j, j + 1,
// w from k, k + 1 (periodic), written (u, v, w) per probe
template <class T>
__global__ void k_probe(const int* __restrict__ ijk, int n, int ny, int nz, const T* __restrict__ u,
                        const T* __restrict__ v, const T* __restrict__ w, T* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int i = ijk[3 * q], j = ijk[3 * q + 1], k = ijk[3 * q + 2];
  const int jp = j + 1 == ny ? 0 : j + 1, kp = k + 1 == nz ? 0 : k + 1;
  const size_t P = (size_t)ny * nz, c = (size_t)i * P + (size_t)j * nz + k;
  out[3 * q] = (T)0.5 * (u[c] + u[c + P]);
  out[3 * q + 1] = (T)0.5 * (v[c] + v[(size_t)i * P + (size_t)jp * nz + k]);
  out[3 * q + 2] = (T)0.5 * (w[c] + w[(size_t)i * P + (size_t)j * nz + kp]);
}

// bounded wait on an mbarrier that nothing completes: at most `spins`
// try-wait rounds, then the time-out goes to the flag as in the solver's kernels
__global__ void k_wait_selftest(uint32_t spins, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (uint32_t it = 0; it < spins && !done; ++it) done = mbar_try_wait(&bar, 0);
    if (!done) atomicOr(flag, ERR_TIMEOUT);
  }
}

}  // namespace

namespace {
// pieces of a member's step for the batched ensemble: the step's start
// (dt, implicit-factor tables), its explicit stage (batched across the
// members), the rest of its head (inflow, outflow, implicit factors), its
// tail (forcing, structure joined, pressure, projection)
template <class T>
void record_pre(ibm_state* s, int cur) {
  Fields<T>& f = fields<T>(s);
  launch_begin_step(s->c, f, s->stream);
  launch_af_tables(s->c, f, s->stream);
  (void)cur;
}
template <class T>
void record_post(ibm_state* s, int cur) {
  Fields<T>& f = fields<T>(s);
  launch_inflow(s->c, f, cur, s->stream);
  launch_outflow(s->c, f, cur, s->stream);
  launch_af(s->c, f, cur, s->stream);
}
template <class T>
void record_tail_joined(ibm_state* s, int cur) {
  const bool join = record_tail_body<T>(s, cur);
  launch_speed_check(s->c, fields<T>(s), s->stream);
  if (join) cudaStreamWaitEvent(s->stream, s->ev_join, 0);
}

// capture one piece of a member's step into a graph
template <class T>
cudaError_t capture_piece(ibm_state* s, int piece, int cur, cudaGraph_t* g) {
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  if (piece == 0) record_pre<T>(s, cur);
  else if (piece == 1) record_post<T>(s, cur);
  else record_tail_joined<T>(s, cur);
  return cudaStreamEndCapture(s->stream, g);
}

cudaError_t member_piece(ibm_state* s, int piece, int cur, cudaGraph_t* g) {
  return s->precision == IBM_FP64 ? capture_piece<double>(s, piece, cur, g) : capture_piece<float>(s, piece, cur, g);
}

// the case table of the members of one field precision at offset `off`,
// uploaded to device memory; returns the number of blocks in *total
template <class T>
cudaError_t build_cases(const std::vector<ibm_state*>& ms, int off, void** dtab, int* ncases, int* total) {
  std::vector<RhsCase<T>> tab;
  int first = 0;
  for (ibm_state* m : ms) {
    if ((m->precision == IBM_FP64) != std::is_same<T, double>::value) continue;
    RhsCase<T> e = rhs_case<T>(m->c, fields<T>(m), (m->cur + off) & 1);
    e.first = first;
    first += e.gx * e.gy * e.gz;
    tab.push_back(e);
  }
  *ncases = (int)tab.size();
  *total = first;
  *dtab = nullptr;
  if (tab.empty()) return cudaSuccess;
  cudaError_t err = cudaMalloc(dtab, tab.size() * sizeof(RhsCase<T>));
  if (err != cudaSuccess) return err;
  return cudaMemcpy(*dtab, tab.data(), tab.size() * sizeof(RhsCase<T>), cudaMemcpyHostToDevice);
}

// the persistent launch over a case table, captured on `st` into a graph
template <class T>
cudaError_t cases_graph(const void* dtab, int ncases, int total, cudaStream_t st, cudaGraph_t* g) {
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = std::max(1, std::min(total, 8 * std::max(sms, 1)));
  launch_rhs_cases<T>((const RhsCase<T>*)dtab, ncases, total, blocks, st);
  return cudaStreamEndCapture(st, g);
}

int create_impl(const ibm_grid* g, const ibm_domain* d, double re, const ibm_bodies* b,
                const ibm_options* o, const ibm_slab* sl, void* workspace, size_t workspace_bytes,
                ibm_state** out);

// ------------------------------------------------------------------ x slabs
// bit of a phase in the allowed-phase mask
constexpr int slab_bit(int phase) { return 1 << phase; }

// overlap planes needed at this viscosity, spacing and step (see ibm_slab_ghosts)
int slab_min_ghosts(double nu, double h, double dt) {
  const double r = nu * dt / (2.0 * h * h);
  const double rho = std::exp(-2.0 * std::asinh(0.5 / std::sqrt(r)));
  int H = (int)std::ceil(std::log(1e-17) / std::log(rho));
  if (!(H >= 1)) H = 1;
  return H + 4;
}

// doubles in one half of the overlap exchange: u, v, w with ghosts + 1
// planes, p with ghosts planes. The advection history N^{n-1} is not
// exchanged: each rank computes it from the refreshed velocity, exact except
// next to the window's ends, where it only disturbs planes that the implicit
// x factor's decay keeps away from the owned ones (and that the next refresh
// replaces)
size_t slab_halo_half(size_t P, int g) { return (size_t)(4 * g + 3) * P; }

int slab_setup(ibm_state* s, const ibm_slab& sl, int nx_global) {
  SlabDev& sd = s->slab;
  int x0, nxw;
  sd.gL = slab_window(sl, &x0, &nxw);
  sd.nranks = sl.nranks;
  sd.rank = sl.rank;
  sd.x_begin = sl.x_begin;
  sd.x_end = sl.x_end;
  sd.nx_global = nx_global;
  sd.n = sl.x_end - sl.x_begin;
  sd.g = sl.ghosts;
  sd.gR = sl.rank < sl.nranks - 1 ? sl.ghosts : 0;
  sd.first_phys = sl.rank == 0;
  sd.last_phys = sl.rank == sl.nranks - 1;
  const Consts& c = s->c;
  const size_t P = plane(c), PT = poisson_modes(c);
  if (cudaMalloc(&sd.tab, (size_t)sd.n * PT * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sd.green, 6 * PT * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sd.scr, (size_t)sd.n * P * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IBM_ENOMEM;
  }
  slab_tables(c, sd, s->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->stream));
  s->slab_allowed = slab_bit(IBM_SLAB_INIT) | slab_bit(IBM_SLAB_FORCE);
  return IBM_OK;
}

// forward (and, applied again, inverse) transforms of phi in y and z
void slab_transforms(ibm_state* s, bool inverse) {
  Fields<double>& f = s->fd;
  if (launch_dht2d(s->c, f, s->stream)) return;
  if (!inverse) {
    launch_dht_y(s->c, f, s->stream);
    launch_dht_z(s->c, f, s->stream);
  } else {
    launch_dht_z(s->c, f, s->stream);
    launch_dht_y(s->c, f, s->stream);
  }
}

// device-to-device copy of `planes` planes starting at plane i0 of a field
cudaError_t copy_planes(double* dst, const double* src, int i0, int planes, size_t P, bool to_field,
                        cudaStream_t st) {
  if (planes <= 0) return cudaSuccess;
  const size_t bytes = (size_t)planes * P * sizeof(double);
  return to_field ? cudaMemcpyAsync(dst + (size_t)i0 * P, src, bytes, cudaMemcpyDeviceToDevice, st)
                  : cudaMemcpyAsync(dst, src + (size_t)i0 * P, bytes, cudaMemcpyDeviceToDevice, st);
}

int slab_phase_impl(ibm_state* s, int phase, double dt, const double* recv, double* send) {
  Fields<double>& f = s->fd;
  const Consts& c = s->c;
  const SlabDev& sd = s->slab;
  cudaStream_t st = s->stream;
  const size_t P = plane(c);
  const int g = sd.g, n = sd.n, gL = sd.gL;
  switch (phase) {
    case IBM_SLAB_INIT:
      launch_div<double>(c, f, s->cur, true, st);
      slab_transforms(s, false);
      slab_local_solve(c, sd, f.phi, send, st);
      s->slab_initial = true;
      s->slab_allowed = slab_bit(IBM_SLAB_REDUCE);
      break;
    case IBM_SLAB_FORCE: {
      if (!(dt > 0) || sd.g < (sd.nranks > 1 ? slab_min_ghosts(c.nu, c.h, dt) : 0)) return IBM_EINVAL;
      if (dt != s->last_dt_fixed) {
        double two[2] = {dt, s->cfl};
        CK(cudaMemcpyAsync(&f.prm->dt_fixed, two, sizeof(two), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        s->last_dt_fixed = dt;
      }
      launch_begin_step(c, f, st);
      launch_af_tables(c, f, st);
      launch_rhs(c, f, s->cur, st);
      launch_outflow(c, f, s->cur, st);
      launch_af(c, f, s->cur, st);
      launch_ib(c, f, s->mk, s->fl, s->cur, st);
      slab_pack_force(c, sd, s->fl, f.qpart, outflow_blocks(c), send, st);
      s->slab_initial = false;
      s->slab_allowed = slab_bit(IBM_SLAB_SOLVE);
      break;
    }
    case IBM_SLAB_SOLVE:
      slab_unpack_force(c, f.prm, s->fl, recv, st);
      if (s->fl.nv) {   // beside the divergence, transforms and solves; joined in GHOSTS
        CK(cudaEventRecord(s->ev_fork, st));
        CK(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
        launch_flag(f.prm, s->fl, false, s->side);
        CK(cudaEventRecord(s->ev_join, s->side));
      }
      launch_div<double>(c, f, s->cur, false, st);
      slab_transforms(s, false);
      slab_local_solve(c, sd, f.phi, send, st);
      s->slab_allowed = slab_bit(IBM_SLAB_REDUCE);
      break;
    case IBM_SLAB_REDUCE:
      slab_correct(c, sd, f.phi, recv, st);
      slab_transforms(s, true);
      CK(copy_planes(send, f.phi, gL, 1, P, false, st));
      CK(copy_planes(send + P, f.phi, gL + n - 1, 1, P, false, st));
      s->slab_allowed = slab_bit(IBM_SLAB_PROJECT);
      break;
    case IBM_SLAB_PROJECT: {
      if (sd.gL > 0) CK(copy_planes(f.phi, recv, gL - 1, 1, P, true, st));
      if (sd.gR > 0) CK(copy_planes(f.phi, recv + P, gL + n, 1, P, true, st));
      launch_project<double>(c, f, s->cur, s->slab_initial, st);
      s->cur ^= 1;
      const int cur = s->cur;
      double* arr[4] = {f.u[cur], f.v[cur], f.w[cur], f.p};
      const size_t half = slab_halo_half(P, g);
      if (sd.gL > 0) {   // to rank - 1: its right overlap, our planes [gL, gL + g] (p: g planes)
        size_t off = 0;
        for (int a = 0; a < 4; ++a) {
          const int planes = a < 3 ? g + 1 : g;
          CK(copy_planes(send + off, arr[a], gL, planes, P, false, st));
          off += (size_t)planes * P;
        }
      }
      if (sd.gR > 0) {   // to rank + 1: its left overlap, our last g owned planes
        size_t off = half;
        for (int a = 0; a < 4; ++a) {
          CK(copy_planes(send + off, arr[a], gL + n - g, g, P, false, st));
          off += (size_t)g * P;
        }
      }
      s->slab_initial = false;
      s->slab_allowed = slab_bit(IBM_SLAB_GHOSTS);
      break;
    }
    case IBM_SLAB_GHOSTS: {
      const int cur = s->cur;
      double* arr[4] = {f.u[cur], f.v[cur], f.w[cur], f.p};
      const size_t half = slab_halo_half(P, g);
      if (sd.gL > 0) {   // from rank - 1: g planes per array into planes [0, g)
        size_t off = 0;
        for (int a = 0; a < 4; ++a) {
          CK(copy_planes(arr[a], recv + off, 0, g, P, true, st));
          off += (size_t)g * P;
        }
      }
      if (sd.gR > 0) {   // from rank + 1: planes [nx - g, nx] (p: [nx - g, nx))
        size_t off = half;
        for (int a = 0; a < 4; ++a) {
          const int planes = a < 3 ? g + 1 : g;
          CK(copy_planes(arr[a], recv + off, c.nx - g, planes, P, true, st));
          off += (size_t)planes * P;
        }
      }
      s->slab_allowed = slab_bit(IBM_SLAB_INIT) | slab_bit(IBM_SLAB_FORCE);
      CK(cudaStreamWaitEvent(st, s->ev_join, 0));   // the step's structural update
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(s->hprm, f.prm, sizeof(Params), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const Params& p = *s->hprm;
      if (p.error & ERR_TIMEOUT) return IBM_ETIMEOUT;
      if (p.error & ERR_AF_RANGE) return IBM_EINVAL;
      if (p.error) return IBM_EDIVERGED;
      return IBM_OK;
    }
    default:
      return IBM_EINVAL;
  }
  CK(cudaGetLastError());
  return IBM_OK;
}

size_t slab_send_count(int phase, size_t P, int nv, int g) {
  switch (phase) {
    case IBM_SLAB_INIT:
    case IBM_SLAB_SOLVE: return (size_t)SLAB_LINE * P;
    case IBM_SLAB_FORCE: return 3 * (size_t)nv + 2;
    case IBM_SLAB_REDUCE: return 2 * P;
    case IBM_SLAB_PROJECT: return 2 * slab_halo_half(P, g);
    default: return 0;
  }
}
}  // namespace

extern "C" {

int ibm_slab_ghosts(double re, double h, double dt, int* ghosts) {
  if (!ghosts || !(re > 0) || !(h > 0) || !(dt > 0) || !std::isfinite(re * h * dt)) return IBM_EINVAL;
  *ghosts = slab_min_ghosts(1.0 / re, h, dt);
  return IBM_OK;
}

int ibm_slab_split(int nx, int nranks, int rank, int ghosts, ibm_slab* out) {
  if (!out || nx < 4 || nranks < 1 || nranks > IBM_SLAB_MAX_RANKS || rank < 0 || rank >= nranks || ghosts < 0)
    return IBM_EINVAL;
  const int base = nx / nranks, rem = nx % nranks;
  ibm_slab sl;
  sl.nranks = nranks;
  sl.rank = rank;
  sl.x_begin = rank * base + std::min(rank, rem);
  sl.x_end = sl.x_begin + base + (rank < rem ? 1 : 0);
  sl.ghosts = nranks > 1 ? ghosts : 0;
  ibm_grid g{nx, 4, 4};
  for (int q = 0; q < nranks; ++q) {   // every slab long enough for its overlap
    ibm_slab t = sl;
    t.rank = q;
    t.x_begin = q * base + std::min(q, rem);
    t.x_end = t.x_begin + base + (q < rem ? 1 : 0);
    if (check_slab(&g, nullptr, &t)) return IBM_EINVAL;
  }
  *out = sl;
  return IBM_OK;
}

int ibm_slab_plan(const ibm_grid* grid, int nv, const ibm_slab* sl, int phase, int* xchg, size_t* send_count,
                  size_t* recv_count) {
  if (!grid || !sl || !xchg || !send_count || !recv_count || nv < 0 || grid->ny < 1 || grid->nz < 1 ||
      phase < IBM_SLAB_INIT || phase > IBM_SLAB_GHOSTS || sl->nranks < 1 || sl->nranks > IBM_SLAB_MAX_RANKS ||
      sl->ghosts < 0)
    return IBM_EINVAL;
  const size_t P = (size_t)grid->ny * grid->nz;
  const size_t n = slab_send_count(phase, P, nv, sl->ghosts);
  *send_count = n;
  switch (phase) {
    case IBM_SLAB_INIT:
    case IBM_SLAB_SOLVE:
      *xchg = IBM_XCHG_GATHER;
      *recv_count = n * sl->nranks;
      break;
    case IBM_SLAB_FORCE:
      *xchg = IBM_XCHG_SUM;
      *recv_count = n;
      break;
    case IBM_SLAB_REDUCE:
    case IBM_SLAB_PROJECT:
      *xchg = IBM_XCHG_HALO;
      *recv_count = n;
      break;
    default:
      *xchg = IBM_XCHG_NONE;
      *recv_count = 0;
      break;
  }
  return IBM_OK;
}

int ibm_slab_workspace_bytes(const ibm_grid* g, const ibm_domain* d, const ibm_bodies* b, const ibm_options* o,
                             const ibm_slab* sl, size_t* bytes) {
  if (!bytes || !sl) return IBM_EINVAL;
  ibm_state tmp;
  FlagGeom fg;
  std::vector<double> Xb;
  double bdv;
  Layout L;
  BarMask bm;
  int rc = prepare(g, d, b, o, &tmp, fg, Xb, bdv, L, bm, sl);
  if (rc) return rc;
  *bytes = carve<double>(&tmp, nullptr, L, tmp.fd);
  return IBM_OK;
}

int ibm_slab_phase(ibm_state* s, int phase, double dt, const double* recv, double* send) {
  if (!s || !s->slab_on || phase < IBM_SLAB_INIT || phase > IBM_SLAB_GHOSTS) return IBM_EINVAL;
  if (!(s->slab_allowed & slab_bit(phase))) return IBM_EINVAL;
  const bool needs_recv = phase != IBM_SLAB_INIT && phase != IBM_SLAB_FORCE;
  const bool needs_send = phase != IBM_SLAB_GHOSTS;
  if ((needs_recv && !recv) || (needs_send && !send)) return IBM_EINVAL;
  return slab_phase_impl(s, phase, dt, recv, send);
}


int ibm_check_bounded_wait(unsigned int spins) {
  if (spins < 1 || spins > (1u << 24)) return IBM_EINVAL;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return IBM_ECUDA;
  }
  int h = 0;
  cudaError_t e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>(spins, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IBM_ECUDA;
  }
  return (h & ERR_TIMEOUT) ? IBM_ETIMEOUT : IBM_OK;
}

const char* ibm_strerror(int code) {
  switch (code) {
    case IBM_OK: return "ok";
    case IBM_EINVAL: return "invalid argument";
    case IBM_ENOMEM: return "device workspace missing, too small or not allocatable";
    case IBM_ECUDA: return "CUDA runtime error";
    case IBM_EDIVERGED: return "solution diverged (non-finite velocity or CFL above limit)";
    case IBM_ETIMEOUT: return "bounded device wait ran out";
    case IBM_EIO: return "checkpoint I/O error";
    default: return "unknown status";
  }
}

int ibm_workspace_bytes(const ibm_grid* g, const ibm_domain* d, const ibm_bodies* b,
                        const ibm_options* o, size_t* bytes) {
  if (!bytes) return IBM_EINVAL;
  ibm_state tmp;
  FlagGeom fg;
  std::vector<double> Xb;
  double bdv;
  Layout L;
  BarMask bm;
  int rc = prepare(g, d, b, o, &tmp, fg, Xb, bdv, L, bm);
  if (rc) return rc;
  *bytes = tmp.precision == IBM_FP64 ? carve<double>(&tmp, nullptr, L, tmp.fd)
                                     : carve<float>(&tmp, nullptr, L, tmp.ff);
  return IBM_OK;
}

int ibm_create(const ibm_grid* g, const ibm_domain* d, double re, const ibm_bodies* b,
               const ibm_options* o, void* workspace, size_t workspace_bytes, ibm_state** out) {
  return create_impl(g, d, re, b, o, nullptr, workspace, workspace_bytes, out);
}

int ibm_create_slab(const ibm_grid* g, const ibm_domain* d, double re, const ibm_bodies* b,
                    const ibm_options* o, const ibm_slab* sl, void* workspace, size_t workspace_bytes,
                    ibm_state** out) {
  if (!sl) return IBM_EINVAL;
  return create_impl(g, d, re, b, o, sl, workspace, workspace_bytes, out);
}

}  // extern "C"

namespace {
int create_impl(const ibm_grid* g, const ibm_domain* d, double re, const ibm_bodies* b,
                const ibm_options* o, const ibm_slab* sl, void* workspace, size_t workspace_bytes,
                ibm_state** out) {
  if (!out || !(re > 0)) return IBM_EINVAL;
  *out = nullptr;
  std::unique_ptr<ibm_state> s(new (std::nothrow) ibm_state());
  if (!s) return IBM_ENOMEM;
  FlagGeom fg;
  std::vector<double> Xb;
  double bdv = 0;
  Layout L;
  BarMask bm;
  int rc = prepare(g, d, b, o, s.get(), fg, Xb, bdv, L, bm, sl);
  if (rc) return rc;
  s->slab_on = sl != nullptr;
  s->c.nu = 1.0 / re;
  s->c.f_nu = (float)s->c.nu;
  const size_t need = s->precision == IBM_FP64 ? carve<double>(s.get(), nullptr, L, s->fd)
                                               : carve<float>(s.get(), nullptr, L, s->ff);
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace & 255)) return IBM_ENOMEM;
    s->ws = workspace;
    s->own_ws = false;
  } else {
    if (cudaMalloc(&s->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return IBM_ENOMEM;
    }
    s->own_ws = true;
  }
  s->ws_bytes = need;
  if (s->precision == IBM_FP64) carve<double>(s.get(), s->ws, L, s->fd);
  else carve<float>(s.get(), s->ws, L, s->ff);
  if (o && o->stream) {
    s->stream = (cudaStream_t)o->stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (s->own_ws) cudaFree(s->ws);
      return IBM_ECUDA;
    }
    s->own_stream = true;
  }
  if (cudaMallocHost(&s->hprm, sizeof(Params)) != cudaSuccess) {
    cudaGetLastError();
    ibm_destroy(s.release());
    return IBM_ECUDA;
  }
  rc = s->precision == IBM_FP64 ? init_state<double>(s.get(), o, fg, Xb, bdv, bm)
                                : init_state<float>(s.get(), o, fg, Xb, bdv, bm);
  if (!rc && sl) rc = slab_setup(s.get(), *sl, g->nx);
  if (rc) {
    ibm_destroy(s.release());
    return rc;
  }
  *out = s.release();
  return IBM_OK;
}
}  // namespace

extern "C" {

int ibm_step(ibm_state* s, double dt, int nsteps) {
  if (!s || nsteps < 0 || s->slab_on) return IBM_EINVAL;
  return s->precision == IBM_FP64 ? step_impl<double>(s, dt, nsteps) : step_impl<float>(s, dt, nsteps);
}

int ibm_sync(ibm_state* s) {
  if (!s) return IBM_EINVAL;
  CK(cudaStreamSynchronize(s->stream));
  return IBM_OK;
}

int ibm_flag_state(ibm_state* s, double* X, double* V, double* F, size_t n) {
  if (!s || !X) return IBM_EINVAL;
  if (n != (size_t)s->fl.nv || n == 0) return IBM_EINVAL;
  cudaStream_t st = s->stream;
  CK(cudaMemcpyAsync(X, s->fl.X, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (V) CK(cudaMemcpyAsync(V, s->fl.V, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (F) CK(cudaMemcpyAsync(F, s->fl.Ff, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

int ibm_stats(ibm_state* s, ibm_stats_t* out) {
  if (!s || !out) return IBM_EINVAL;
  cudaStream_t st = s->stream;
  CK(cudaMemsetAsync(s->dstat, 0, 16 * sizeof(double), st));
  if (s->precision == IBM_FP64) launch_stats<double>(s->c, s->fd, s->cur, s->dstat, st);
  else launch_stats<float>(s->c, s->ff, s->cur, s->dstat, st);
  launch_flag_stats(s->fl, s->dstat + 4, st);
  CK(cudaGetLastError());
  double h[16];
  CK(cudaMemcpyAsync(h, s->dstat, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(s->hprm, s->prm, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const Params& p = *s->hprm;
  std::memset(out, 0, sizeof(*out));
  out->step = p.step;
  out->t = p.t;
  out->dt = p.dt;
  out->cfl = p.dt * p.speed_max / s->c.h;
  out->ke = h[0];
  out->max_div = h[1];
  out->q_in = p.q_in;
  out->q_out = p.q_out;
  out->ib_slip = p.slip_max;
  if (s->fl.nv) {
    for (int e = 0; e < 3; ++e) {
      out->te_mid[e] = h[4 + e];
      out->force[e] = h[7 + e];
    }
    out->max_strain = h[10];
  }
  out->n_sub = p.n_sub;
  out->n_markers = s->mk.nm;
  out->kernels_per_step = s->kernels_per_step;
  return IBM_OK;
}

int ibm_time_stage(ibm_state* s, int stage, int nrep, double* ms) {
  if (!s || !ms || nrep < 1 || stage < IBM_STAGE_STEP || stage > IBM_STAGE_POISSON_X16) return IBM_EINVAL;
  if (stage == IBM_STAGE_STEP && s->slab_on) return IBM_EINVAL;   // a slab state captures no step
  cudaStream_t st = s->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  for (int r = 0; r < nrep; ++r) {
    if (stage == IBM_STAGE_STEP) {
      cudaGraphLaunch(s->exec[GRAPH_HEAD][s->cur], st);
      cudaGraphLaunch(s->exec[GRAPH_TAIL][s->cur], st);
      s->cur ^= 1;
    } else if (s->precision == IBM_FP64) {
      launch_stage<double>(s, stage);
    } else {
      launch_stage<float>(s, stage);
    }
  }
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaError_t e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  CK(cudaGetLastError());
  *ms = (double)t / nrep;
  return IBM_OK;
}

// doubles that fit in the FP32 scratch buffer e[0] (one field of floats)
static size_t stage_capacity(const ibm_state* s) {
  const Consts& c = s->c;
  return (size_t)(c.nx + 1) * c.ny * c.nz / 2;
}

static int field_ptr(ibm_state* s, int which, void** ptr, size_t* n) {
  const Consts& c = s->c;
  const size_t NF = (size_t)(c.nx + 1) * c.ny * c.nz, NP = (size_t)c.nx * c.ny * c.nz;
  const bool d = s->precision == IBM_FP64;
  switch (which) {
    case IBM_FIELD_U: *ptr = d ? (void*)s->fd.u[s->cur] : (void*)s->ff.u[s->cur]; *n = NF; break;
    case IBM_FIELD_V: *ptr = d ? (void*)s->fd.v[s->cur] : (void*)s->ff.v[s->cur]; *n = NF; break;
    case IBM_FIELD_W: *ptr = d ? (void*)s->fd.w[s->cur] : (void*)s->ff.w[s->cur]; *n = NF; break;
    case IBM_FIELD_P: *ptr = d ? (void*)s->fd.p : (void*)s->ff.p; *n = NP; break;
    default: return IBM_EINVAL;
  }
  return IBM_OK;
}

int ibm_get_field(ibm_state* s, int which, double* host, size_t n) {
  if (!s || !host) return IBM_EINVAL;
  void* ptr;
  size_t cnt;
  if (field_ptr(s, which, &ptr, &cnt) || cnt != n) return IBM_EINVAL;
  if (s->precision == IBM_FP64) return download_field<double>(s->stream, host, (double*)ptr, n);
  // staging: the implicit-factor scratch e[0..2] (contiguous, idle between steps)
  return download_f32_staged(s->stream, host, (const float*)ptr, n, (double*)s->ff.e[0],
                             stage_capacity(s));
}

int ibm_set_field(ibm_state* s, int which, const double* host, size_t n) {
  if (!s || !host) return IBM_EINVAL;
  void* ptr;
  size_t cnt;
  if (field_ptr(s, which, &ptr, &cnt) || cnt != n) return IBM_EINVAL;
  if (s->precision == IBM_FP64) return upload_field<double>(s->stream, (double*)ptr, host, n);
  return upload_f32_staged(s->stream, (float*)ptr, host, n, (double*)s->ff.e[0], stage_capacity(s));
}

int ibm_plane_device(ibm_state* s, int i, void** u, void** v, void** w) {
  if (!s || !u || !v || !w || i < 0 || i > s->c.nx) return IBM_EINVAL;
  const size_t off = (size_t)i * s->c.ny * s->c.nz;
  if (s->precision == IBM_FP64) {
    *u = s->fd.u[s->cur] + off;
    *v = s->fd.v[s->cur] + off;
    *w = s->fd.w[s->cur] + off;
  } else {
    *u = s->ff.u[s->cur] + off;
    *v = s->ff.v[s->cur] + off;
    *w = s->ff.w[s->cur] + off;
  }
  return IBM_OK;
}

int ibm_probes_set(ibm_state* s, const int* ijk, int n) {
  if (!s || n < 0 || n > (1 << 22) || (n > 0 && !ijk)) return IBM_EINVAL;
  for (int q = 0; q < n; ++q)
    if (ijk[3 * q] < 0 || ijk[3 * q] >= s->c.nx || ijk[3 * q + 1] < 0 || ijk[3 * q + 1] >= s->c.ny ||
        ijk[3 * q + 2] < 0 || ijk[3 * q + 2] >= s->c.nz)
      return IBM_EINVAL;
  if (s->probes) {
    cudaStreamSynchronize(s->stream);
    cudaFree(s->probes);
    s->probes = nullptr;
    s->nprobe = 0;
  }
  if (n == 0) return IBM_OK;
  if (cudaMalloc(&s->probes, (size_t)3 * n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return IBM_ENOMEM;
  }
  if (cudaMemcpy(s->probes, ijk, (size_t)3 * n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return IBM_ECUDA;
  s->nprobe = n;
  return IBM_OK;
}

int ibm_probe_sample(ibm_state* s, void* dst) {
  if (!s || !dst || s->nprobe == 0) return IBM_EINVAL;
  const int n = s->nprobe, nb = (n + 255) / 256;
  if (s->precision == IBM_FP64)
    k_probe<double><<<nb, 256, 0, s->stream>>>(s->probes, n, s->c.ny, s->c.nz, s->fd.u[s->cur],
                                               s->fd.v[s->cur], s->fd.w[s->cur], (double*)dst);
  else
    k_probe<float><<<nb, 256, 0, s->stream>>>(s->probes, n, s->c.ny, s->c.nz, s->ff.u[s->cur],
                                              s->ff.v[s->cur], s->ff.w[s->cur], (float*)dst);
  return cudaGetLastError() == cudaSuccess ? IBM_OK : IBM_ECUDA;
}

int ibm_get_plane(ibm_state* s, int i, double* u, double* v, double* w) {
  if (!s || !u || !v || !w || i < 0 || i > s->c.nx) return IBM_EINVAL;
  void* p[3];
  int rc = ibm_plane_device(s, i, &p[0], &p[1], &p[2]);
  if (rc) return rc;
  const size_t P = (size_t)s->c.ny * s->c.nz;
  double* out[3] = {u, v, w};
  for (int q = 0; q < 3; ++q) {
    rc = s->precision == IBM_FP64 ? download_field<double>(s->stream, out[q], (double*)p[q], P)
                                  : download_field<float>(s->stream, out[q], (float*)p[q], P);
    if (rc) return rc;
  }
  return IBM_OK;
}

int ibm_inflow_planes(ibm_state* s, void** u, void** v, void** w) {
  if (!s || !u || !v || !w || !s->inflow) return IBM_EINVAL;
  const size_t P = (size_t)s->c.ny * s->c.nz;
  char* base = s->precision == IBM_FP64 ? (char*)s->fd.inflow : (char*)s->ff.inflow;
  const size_t e = s->precision == IBM_FP64 ? 8 : 4;
  *u = base;
  *v = base + P * e;
  *w = base + 2 * P * e;
  return IBM_OK;
}

int ibm_set_inflow(ibm_state* s, const double* u, const double* v, const double* w) {
  if (!s || !u || !v || !w || !s->inflow) return IBM_EINVAL;
  const size_t P = (size_t)s->c.ny * s->c.nz;
  const double* src[3] = {u, v, w};
  for (int q = 0; q < 3; ++q) {
    int rc = s->precision == IBM_FP64
                 ? upload_field<double>(s->stream, s->fd.inflow + q * P, src[q], P)
                 : upload_field<float>(s->stream, s->ff.inflow + q * P, src[q], P);
    if (rc) return rc;
  }
  return IBM_OK;
}

int ibm_marker_count(const ibm_state* s, size_t* n) {
  if (!s || !n) return IBM_EINVAL;
  *n = (size_t)s->mk.nm;
  return IBM_OK;
}

int ibm_get_markers(ibm_state* s, double* X, size_t n) {
  if (!s || !X || n != (size_t)s->mk.nm) return IBM_EINVAL;
  cudaStream_t st = s->stream;
  if (s->mk.nf) CK(cudaMemcpyAsync(X, s->fl.X, 3 * (size_t)s->mk.nf * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (s->mk.nb)
    CK(cudaMemcpyAsync(X + 3 * (size_t)s->mk.nf, s->mk.Xb, 3 * (size_t)s->mk.nb * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

// ------------------------------------------------------------------ checkpoints
// File: a fixed header (magic, version, precision, grid, domain, viscosity,
// body parameters, marker counts, element size), the device Params block,
// then u, v, w (current buffer), p, N^{n-1} (three components) in the
// state's precision, the CFL partial maxima, then the flag X, V, F in FP64. Everything the next
// step reads is in the file; scratch (transform buffers, implicit-factor
// ping-pong buffers) and tables rebuilt at creation are not.
namespace {
struct CkptHeader {
  char magic[8];
  int version, precision, nx, ny, nz, nf, nb, elem, inflow, bar_forcing;
  double lx, ly, lz, nu;
  double body[12];
  long long params_bytes;
};

void fill_header(const ibm_state* s, CkptHeader& h) {
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "IBMCKPT1", 8);
  h.version = 1;
  h.precision = s->precision;
  h.nx = s->c.nx;
  h.ny = s->c.ny;
  h.nz = s->c.nz;
  h.nf = s->mk.nf;
  h.nb = s->mk.nb;
  h.elem = s->precision == IBM_FP64 ? 8 : 4;
  h.inflow = s->inflow ? 1 : 0;
  h.bar_forcing = s->bar_forcing;
  h.lx = s->c.lx;
  h.ly = s->c.ly;
  h.lz = s->c.lz;
  h.nu = s->c.nu;
  const ibm_bodies& b = s->bodies;
  const double body[12] = {(double)b.bars_on, b.bar_x,   b.bar_mesh,  b.bar_width,
                           (double)b.flag_on, b.flag_x_le, b.flag_len, b.flag_span,
                           b.mass_ratio,      b.bending, b.pitch0,    b.stretch};
  std::memcpy(h.body, body, sizeof(body));
  h.params_bytes = (long long)sizeof(Params);
}

// device regions of a checkpoint, in file order: pointer and bytes
std::vector<std::pair<void*, size_t>> ckpt_regions(ibm_state* s) {
  const Consts& c = s->c;
  const size_t NF = (size_t)(c.nx + 1) * c.ny * c.nz, NP = (size_t)c.nx * c.ny * c.nz;
  std::vector<std::pair<void*, size_t>> r;
  r.push_back({s->prm, sizeof(Params)});
  auto add = [&](auto& f) {
    const size_t e = sizeof(*f.p);
    r.push_back({f.u[s->cur], NF * e});
    r.push_back({f.v[s->cur], NF * e});
    r.push_back({f.w[s->cur], NF * e});
    r.push_back({f.p, NP * e});
    for (int q = 0; q < 3; ++q) r.push_back({f.n[q], NF * e});
    // per-block maxima of the CFL speed from the last projection: the next
    // step's dt in CFL mode
    r.push_back({f.partial, (size_t)f.n_partial * sizeof(double)});
    // prescribed inflow planes (pending and current levels)
    if (f.inflow) r.push_back({f.inflow, 8 * (size_t)c.ny * c.nz * e});
  };
  if (s->precision == IBM_FP64) add(s->fd);
  else add(s->ff);
  if (s->fl.nv) {
    const size_t b = 3 * (size_t)s->fl.nv * sizeof(double);
    r.push_back({s->fl.X, b});
    r.push_back({s->fl.V, b});
    r.push_back({s->fl.Ff, b});
  }
  return r;
}

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) std::fclose(f);
  }
};
}  // namespace

int ibm_save(ibm_state* s, const char* path) {
  if (!s || !path) return IBM_EINVAL;
  CK(cudaStreamSynchronize(s->stream));
  CkptHeader h;
  fill_header(s, h);
  std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "wb"));
  if (!f) return IBM_EIO;
  if (std::fwrite(&h, sizeof(h), 1, f.get()) != 1) return IBM_EIO;
  std::vector<char> buf;
  for (auto& reg : ckpt_regions(s)) {
    buf.resize(reg.second);
    CK(cudaMemcpyAsync(buf.data(), reg.first, reg.second, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (std::fwrite(buf.data(), 1, reg.second, f.get()) != reg.second) return IBM_EIO;
  }
  if (std::fflush(f.get()) != 0) return IBM_EIO;
  return IBM_OK;
}

int ibm_load(ibm_state* s, const char* path) {
  if (!s || !path) return IBM_EINVAL;
  std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "rb"));
  if (!f) return IBM_EIO;
  CkptHeader h, mine;
  if (std::fread(&h, sizeof(h), 1, f.get()) != 1) return IBM_EIO;
  fill_header(s, mine);
  if (std::memcmp(h.magic, mine.magic, 8) != 0 || h.version != mine.version) return IBM_EIO;
  // a checkpoint of a different problem: refuse before touching the state
  if (std::memcmp(&h, &mine, sizeof(h)) != 0) return IBM_EINVAL;
  const auto regs = ckpt_regions(s);
  std::vector<std::vector<char>> bufs(regs.size());
  for (size_t q = 0; q < regs.size(); ++q) {
    bufs[q].resize(regs[q].second);
    if (std::fread(bufs[q].data(), 1, regs[q].second, f.get()) != regs[q].second) return IBM_EIO;
  }
  char extra;
  if (std::fread(&extra, 1, 1, f.get()) != 0) return IBM_EIO;   // trailing bytes
  CK(cudaStreamSynchronize(s->stream));
  for (size_t q = 0; q < regs.size(); ++q)
    CK(cudaMemcpyAsync(regs[q].first, bufs[q].data(), regs[q].second, cudaMemcpyHostToDevice,
                       s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->last_dt_fixed = -2.0;   // the time-step mode travels in Params; re-send on the next step
  return IBM_OK;
}

void ibm_destroy(ibm_state* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (int k = 0; k < GRAPH_KINDS; ++k)
    for (int q = 0; q < 2; ++q) {
      if (s->exec[k][q]) cudaGraphExecDestroy(s->exec[k][q]);
      if (s->graph[k][q]) cudaGraphDestroy(s->graph[k][q]);
    }
  if (s->own_ws && s->ws) cudaFree(s->ws);
  if (s->probes) cudaFree(s->probes);
  if (s->slab.tab) cudaFree(s->slab.tab);
  if (s->slab.green) cudaFree(s->slab.green);
  if (s->slab.scr) cudaFree(s->slab.scr);
  if (s->hprm) cudaFreeHost(s->hprm);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->side2) cudaStreamDestroy(s->side2);
  if (s->ev_fork2) cudaEventDestroy(s->ev_fork2);
  if (s->ev_join2) cudaEventDestroy(s->ev_join2);
  cudaGetLastError();
  delete s;
}

// ------------------------------------------------------------------ ensembles
struct ibm_ensemble {
  std::vector<ibm_state*> members;
  // [kind][offset]: every member runs its graph of that kind for buffer
  // parity (its parity at creation + offset) & 1
  cudaGraphExec_t exec[GRAPH_KINDS][2] = {};
  int par = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // batched explicit stage: case tables per offset (FP32-field and FP64
  // members), device memory owned by the ensemble
  void* table[2][2] = {};
};



static int ensemble_set_dt(ibm_state* s, double dt, cudaStream_t st) {
  const double mode = dt > 0 ? dt : -1.0;
  if (mode != s->last_dt_fixed) {
    double two[2] = {mode, s->cfl};
    Params* prm = s->prm;
    CK(cudaMemcpyAsync(&prm->dt_fixed, two, sizeof(two), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    s->last_dt_fixed = mode;
  }
  return IBM_OK;
}

int ibm_ensemble_create(ibm_state* const* members, int n, void* stream, ibm_ensemble** out) {
  if (!members || n < 1 || !out) return IBM_EINVAL;
  *out = nullptr;
  std::unique_ptr<ibm_ensemble> e(new (std::nothrow) ibm_ensemble());
  if (!e) return IBM_ENOMEM;
  for (int q = 0; q < n; ++q) {
    if (!members[q] || !members[q]->graph[GRAPH_MID][0] || !members[q]->graph[GRAPH_MID][1])
      return IBM_EINVAL;
    for (int r = 0; r < q; ++r)
      if (members[r] == members[q]) return IBM_EINVAL;
    e->members.push_back(members[q]);
    CK(cudaStreamSynchronize(members[q]->stream));
  }
  if (stream) {
    e->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    e->own_stream = true;
  }
  // one parent graph per graph kind and parity offset: member q runs its graph
  // of that kind for buffer parity (cur_q + offset) & 1, all members as
  // independent branches
  for (int kind = 0; kind < GRAPH_KINDS; ++kind)
    for (int off = 0; off < 2; ++off) {
      cudaGraph_t parent;
      CK(cudaGraphCreate(&parent, 0));
      for (ibm_state* m : e->members) {
        cudaGraphNode_t node;
        cudaError_t err = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0,
                                                     m->graph[kind][(m->cur + off) & 1]);
        if (err != cudaSuccess) {
          cudaGraphDestroy(parent);
          cudaGetLastError();
          ibm_ensemble_destroy(e.release());
          return IBM_ECUDA;
        }
      }
      cudaError_t err = cudaGraphInstantiate(&e->exec[kind][off], parent, 0);
      cudaGraphDestroy(parent);
      if (err != cudaSuccess) {
        cudaGetLastError();
        ibm_ensemble_destroy(e.release());
        return IBM_ECUDA;
      }
    }
  *out = e.release();
  return IBM_OK;
}

int ibm_ensemble_create_batched(ibm_state* const* members, int n, void* stream, ibm_ensemble** out) {
  if (!members || n < 1 || !out) return IBM_EINVAL;
  *out = nullptr;
  std::unique_ptr<ibm_ensemble> e(new (std::nothrow) ibm_ensemble());
  if (!e) return IBM_ENOMEM;
  for (int q = 0; q < n; ++q) {
    if (!members[q] || !members[q]->graph[GRAPH_MID][0]) return IBM_EINVAL;
    for (int r = 0; r < q; ++r)
      if (members[r] == members[q]) return IBM_EINVAL;
    e->members.push_back(members[q]);
    CK(cudaStreamSynchronize(members[q]->stream));
  }
  if (stream) {
    e->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    e->own_stream = true;
  }
  // member pieces [member][piece][parity] and the batched explicit stage
  // [offset][precision: 0 FP32 fields, 1 FP64]
  std::vector<std::array<std::array<cudaGraph_t, 2>, 3>> pieces(n);
  cudaGraph_t kg[2][2] = {};
  int nc[2][2] = {}, tot[2][2] = {};
  auto fail = [&](cudaError_t err) {
    for (auto& m : pieces)
      for (auto& pc : m)
        for (cudaGraph_t g : pc)
          if (g) cudaGraphDestroy(g);
    for (auto& a : kg)
      for (cudaGraph_t g : a)
        if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ibm_ensemble_destroy(e.release());
    return err == cudaErrorMemoryAllocation ? IBM_ENOMEM : IBM_ECUDA;
  };
  for (int q = 0; q < n; ++q)
    for (int pc = 0; pc < 3; ++pc)
      for (int par = 0; par < 2; ++par) {
        pieces[q][pc][par] = nullptr;
        cudaError_t err = member_piece(e->members[q], pc, par, &pieces[q][pc][par]);
        if (err != cudaSuccess) return fail(err);
      }
  for (int off = 0; off < 2; ++off) {
    cudaError_t err = build_cases<float>(e->members, off, &e->table[off][0], &nc[off][0], &tot[off][0]);
    if (err == cudaSuccess)
      err = build_cases<double>(e->members, off, &e->table[off][1], &nc[off][1], &tot[off][1]);
    if (err == cudaSuccess && nc[off][0])
      err = cases_graph<float>(e->table[off][0], nc[off][0], tot[off][0], e->stream, &kg[off][0]);
    if (err == cudaSuccess && nc[off][1])
      err = cases_graph<double>(e->table[off][1], nc[off][1], tot[off][1], e->stream, &kg[off][1]);
    if (err != cudaSuccess) return fail(err);
  }
  // parent graphs: head = pre -> batched explicit stage -> post;
  // mid = tail -> pre (other parity) -> batched stage -> post; tail = tail
  for (int kind = 0; kind < GRAPH_KINDS; ++kind)
    for (int off = 0; off < 2; ++off) {
      cudaGraph_t parent;
      CK(cudaGraphCreate(&parent, 0));
      cudaError_t err = cudaSuccess;
      std::vector<cudaGraphNode_t> pre(n), tails(n);
      const int hoff = kind == GRAPH_MID ? off ^ 1 : off;   // offset of the head part
      for (int q = 0; q < n && err == cudaSuccess; ++q) {
        ibm_state* m = e->members[q];
        const int pt = (m->cur + off) & 1, ph = (m->cur + hoff) & 1;
        if (kind != GRAPH_HEAD)
          err = cudaGraphAddChildGraphNode(&tails[q], parent, nullptr, 0, pieces[q][2][pt]);
        if (err == cudaSuccess && kind != GRAPH_TAIL)
          err = cudaGraphAddChildGraphNode(&pre[q], parent, kind == GRAPH_MID ? &tails[q] : nullptr,
                                           kind == GRAPH_MID ? 1 : 0, pieces[q][0][ph]);
      }
      if (kind != GRAPH_TAIL) {
        cudaGraphNode_t kn[2] = {};
        for (int t = 0; t < 2 && err == cudaSuccess; ++t) {
          if (!kg[hoff][t]) continue;
          std::vector<cudaGraphNode_t> deps;
          for (int q = 0; q < n; ++q)
            if ((e->members[q]->precision == IBM_FP64) == (t == 1)) deps.push_back(pre[q]);
          err = cudaGraphAddChildGraphNode(&kn[t], parent, deps.data(), deps.size(), kg[hoff][t]);
        }
        for (int q = 0; q < n && err == cudaSuccess; ++q) {
          ibm_state* m = e->members[q];
          cudaGraphNode_t post;
          const cudaGraphNode_t dep = kn[m->precision == IBM_FP64 ? 1 : 0];
          err = cudaGraphAddChildGraphNode(&post, parent, &dep, 1, pieces[q][1][(m->cur + hoff) & 1]);
        }
      }
      if (err == cudaSuccess) err = cudaGraphInstantiate(&e->exec[kind][off], parent, 0);
      cudaGraphDestroy(parent);
      if (err != cudaSuccess) return fail(err);
    }
  for (auto& m : pieces)
    for (auto& pc : m)
      for (cudaGraph_t g : pc) cudaGraphDestroy(g);
  for (auto& a : kg)
    for (cudaGraph_t g : a)
      if (g) cudaGraphDestroy(g);
  *out = e.release();
  return IBM_OK;
}

int ibm_ensemble_step(ibm_ensemble* e, double dt, int nsteps) {
  if (!e || nsteps < 0) return IBM_EINVAL;
  cudaStream_t st = e->stream;
  for (ibm_state* m : e->members) {
    int rc = ensemble_set_dt(m, dt, st);
    if (rc) return rc;
  }
  if (nsteps > 0) {
    CK(cudaGraphLaunch(e->exec[GRAPH_HEAD][e->par], st));
    for (int n = 1; n < nsteps; ++n) {
      CK(cudaGraphLaunch(e->exec[GRAPH_MID][e->par], st));
      e->par ^= 1;
    }
    CK(cudaGraphLaunch(e->exec[GRAPH_TAIL][e->par], st));
    e->par ^= 1;
    if (nsteps & 1)
      for (ibm_state* m : e->members) m->cur ^= 1;
  }
  int result = IBM_OK;
  for (ibm_state* m : e->members)
    CK(cudaMemcpyAsync(m->hprm, m->prm, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (ibm_state* m : e->members) {
    const Params& p = *m->hprm;
    int rc = IBM_OK;
    if (p.error & ERR_TIMEOUT) rc = IBM_ETIMEOUT;
    else if (p.error & ERR_AF_RANGE) rc = IBM_EINVAL;
    else if (p.error) rc = IBM_EDIVERGED;
    else if (nsteps > 0 && p.dt * p.speed_max / m->c.h > m->cfl_limit) rc = IBM_EDIVERGED;
    if (rc && result == IBM_OK) result = rc;
  }
  return result;
}

void ibm_ensemble_destroy(ibm_ensemble* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  for (int k = 0; k < GRAPH_KINDS; ++k)
    for (int q = 0; q < 2; ++q)
      if (e->exec[k][q]) cudaGraphExecDestroy(e->exec[k][q]);
  for (auto& a : e->table)
    for (void* t : a)
      if (t) cudaFree(t);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  cudaGetLastError();
  delete e;
}

}  // extern "C"

// ------------------------------------------------------------------ diagnostics without allocation
// Reduction scratch of ibm_stats_static: a fixed device array in this file
// (host code only ever sees its address through cudaGetSymbolAddress).
namespace {
constexpr int kStatsMaxBlocks = 1 << 16;
constexpr int kStatsScratch = 2 * kStatsMaxBlocks + 16;
__device__ __align__(256) double g_stats_scratch[kStatsScratch];
constexpr int kMaxDevices = 64;
// the array's device address per device, looked up on the first call there;
// concurrent first calls store the same value; stale after cudaDeviceReset
double* g_stats_dev_ptr[kMaxDevices] = {nullptr};

constexpr int kSTK = 32, kSTJ = 8, kSX = 8;   // block tile of the first pass

// first pass: per-block kinetic energy and max |div u| (no atomics)
template <class T>
__global__ void __launch_bounds__(kSTK* kSTJ)
k_stats_blocks(Consts c, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
               double* __restrict__ part) {
  __shared__ double sk[kSTK * kSTJ / 32], sd[kSTK * kSTJ / 32];
  const int k = blockIdx.x * kSTK + threadIdx.x;
  const int j = blockIdx.y * kSTJ + threadIdx.y;
  double ke = 0.0, dmax = 0.0;
  if (k < c.nz && j < c.ny) {
    const int ny = c.ny, nz = c.nz, nx = c.nx;
    const int jp = j == ny - 1 ? 0 : j + 1, kp = k == nz - 1 ? 0 : k + 1;
    const size_t P = (size_t)ny * nz;
    const int i0 = blockIdx.z * kSX, i1 = min(i0 + kSX, nx + 1);
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
  const int tid = threadIdx.y * kSTK + threadIdx.x;
  if ((tid & 31) == 0) {
    sk[tid >> 5] = ke;
    sd[tid >> 5] = dmax;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < kSTK * kSTJ / 32; ++q) {
      a += sk[q];
      b = fmax(b, sd[q]);
    }
    const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[blk] = a;
    part[kStatsMaxBlocks + blk] = b;
  }
}

// second pass: one block reduces the partials in a fixed order
__global__ void k_stats_final(int nblk, double h3, const double* __restrict__ part,
                              double* __restrict__ res) {
  __shared__ double scratch[32];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    a += part[q];
    b = fmax(b, part[kStatsMaxBlocks + q]);
  }
  a = block_sum(a, scratch);
  __syncthreads();
  b = block_max(b, scratch);
  if (threadIdx.x == 0) {
    res[0] = a * h3;
    res[1] = b;
  }
}
}  // namespace

extern "C" int ibm_stats_static(ibm_state* s, ibm_stats_t* out) {
  if (!s || !out) return IBM_EINVAL;
  const Consts& c = s->c;
  const dim3 grid((c.nz + kSTK - 1) / kSTK, (c.ny + kSTJ - 1) / kSTJ, (c.nx + 1 + kSX - 1) / kSX);
  const long long nblk = (long long)grid.x * grid.y * grid.z;
  if (nblk > kStatsMaxBlocks) return IBM_EINVAL;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return IBM_EINVAL;
  if (!g_stats_dev_ptr[dev]) {
    double* ptr = nullptr;
    CK(cudaGetSymbolAddress((void**)&ptr, g_stats_scratch));
    g_stats_dev_ptr[dev] = ptr;
  }
  double* part = g_stats_dev_ptr[dev];
  double* res = part + 2 * kStatsMaxBlocks;
  cudaStream_t st = s->stream;
  if (s->precision == IBM_FP64)
    k_stats_blocks<double><<<grid, dim3(kSTK, kSTJ), 0, st>>>(c, s->fd.u[s->cur], s->fd.v[s->cur],
                                                             s->fd.w[s->cur], part);
  else
    k_stats_blocks<float><<<grid, dim3(kSTK, kSTJ), 0, st>>>(c, s->ff.u[s->cur], s->ff.v[s->cur],
                                                            s->ff.w[s->cur], part);
  k_stats_final<<<1, 1024, 0, st>>>((int)nblk, c.h * c.h * c.h, part, res);
  launch_flag_stats(s->fl, res + 4, st);
  CK(cudaGetLastError());
  double h[16];
  CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(s->hprm, s->prm, sizeof(Params), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const Params& p = *s->hprm;
  std::memset(out, 0, sizeof(*out));
  out->step = p.step;
  out->t = p.t;
  out->dt = p.dt;
  out->cfl = p.dt * p.speed_max / c.h;
  out->ke = h[0];
  out->max_div = h[1];
  out->q_in = p.q_in;
  out->q_out = p.q_out;
  out->ib_slip = p.slip_max;
  if (s->fl.nv) {
    for (int e = 0; e < 3; ++e) {
      out->te_mid[e] = h[4 + e];
      out->force[e] = h[7 + e];
    }
    out->max_strain = h[10];
  }
  out->n_sub = p.n_sub;
  out->n_markers = s->mk.nm;
  out->kernels_per_step = s->kernels_per_step;
  return IBM_OK;
}
