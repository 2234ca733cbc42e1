// Host mesh layer: validation, periodic wrap (Sec. 2.5), node graph, reverse Cuthill-McKee
// renumbering, linear-tetrahedron geometry, and node-centric assembly of the FEM operators of
// Eqs. LHS and RHS_F into SELL-32 arrays.  Runs once per mesh; parallel over rows with OpenMP
// (each row is summed in a fixed order, so results do not depend on the thread count).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <numeric>
#include <unordered_map>

#include "internal.h"

namespace gspm {

int make_params(const gspm_material* m, const gspm_options* o, Params* p) {
  if (!(m->Ms > 0) || !(o->dt > 0) || !(o->alpha >= 0) || !(m->A >= 0)) {
    set_error("material/options: need Ms > 0, A >= 0, dt > 0, alpha >= 0");
    return GSPM_EINVAL;
  }
  p->Ms = m->Ms;
  p->mu0 = m->mu0 > 0 ? m->mu0 : 1.25663706212e-6;
  p->gamma0 = m->gamma0 > 0 ? m->gamma0 : 2.2127615e5;
  p->l_d = m->l_d > 0 ? m->l_d : 1e-9;
  p->scale = p->mu0 * p->Ms * p->Ms;
  p->A_star = 2.0 * m->A / (p->scale * p->l_d * p->l_d);
  p->kappa = 2.0 * m->K1 / p->scale;
  p->dtau = p->gamma0 * p->Ms * o->dt;
  p->alpha = o->alpha;
  p->eps = p->A_star * p->dtau;
  p->C11 = m->C11; p->C12 = m->C12; p->C44 = m->C44;
  p->l100 = m->lambda100; p->l111 = m->lambda111;
  p->me_coef = 3.0 / p->scale;
  for (int i = 0; i < 9; ++i) p->Nd[i] = m->Nd[i];
  // App. D rotation (all zero = identity); must be a proper rotation
  bool zero = true;
  for (int i = 0; i < 9; ++i) zero = zero && m->R[i] == 0.0;
  for (int i = 0; i < 9; ++i) p->R[i] = zero ? (i % 4 == 0 ? 1.0 : 0.0) : m->R[i];
  {
    double err = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double d = 0.0;
        for (int k = 0; k < 3; ++k) d += p->R[3 * i + k] * p->R[3 * j + k];
        err = std::max(err, std::fabs(d - (i == j ? 1.0 : 0.0)));
      }
    const double* R = p->R;
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (err > 1e-12 || std::fabs(det - 1.0) > 1e-12) {
      set_error("material: R is not a proper rotation (R R^T = I, det R = 1 to 1e-12)");
      return GSPM_EINVAL;
    }
  }
  p->rotated = 0;
  for (int i = 0; i < 9; ++i) p->rotated |= p->R[i] != (i % 4 == 0 ? 1.0 : 0.0);
  // stiffness tensor in the mesh axes: C'_ijkl = R_ia R_jb R_kc R_ld C_abcd (cubic C in the
  // crystal axes)
  double Cc[81];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          double v = 0.0;
          if (a == b && c == d) v = a == c ? m->C11 : m->C12;
          else if ((a == c && b == d) || (a == d && b == c)) v = m->C44;
          Cc[((a * 3 + b) * 3 + c) * 3 + d] = v;
        }
  for (int i = 0; i < 81; ++i) {
    const int ii = i / 27, jj = (i / 9) % 3, kk = (i / 3) % 3, ll = i % 3;
    double v = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d)
            v += p->R[3 * ii + a] * p->R[3 * jj + b] * p->R[3 * kk + c] * p->R[3 * ll + d] *
                 Cc[((a * 3 + b) * 3 + c) * 3 + d];
    p->Cm[i] = v;
  }
  // E_ext = C^-1 sigma_ext: rotate sigma_ext into the crystal axes (R^T s R), apply the cubic
  // compliance (closed-form inverse of the normal block; tensor shear strain = sigma / (2 C44)),
  // rotate back (R e R^T)
  const double d = (m->C11 - m->C12) * (m->C11 + 2.0 * m->C12);
  if (!(d != 0.0) || !(m->C44 != 0.0)) {
    set_error("material: singular elastic stiffness");
    return GSPM_EINVAL;
  }
  const double S11 = (m->C11 + m->C12) / d, S12 = -m->C12 / d;
  const double* sv = m->sigma_ext;
  const double sm[3][3] = {{sv[0], sv[5], sv[4]}, {sv[5], sv[1], sv[3]}, {sv[4], sv[3], sv[2]}};
  double sc[3][3], ec[3][3], em[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) v += p->R[3 * a + i] * sm[a][b] * p->R[3 * b + j];
      sc[i][j] = v;
    }
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    ec[i][i] = S11 * sc[i][i] + S12 * (sc[j][j] + sc[k][k]);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j) ec[i][j] = sc[i][j] / (2.0 * m->C44);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) v += p->R[3 * i + a] * ec[a][b] * p->R[3 * j + b];
      em[i][j] = v;
    }
  p->E_ext[0] = em[0][0];
  p->E_ext[1] = em[1][1];
  p->E_ext[2] = em[2][2];
  p->E_ext[3] = em[1][2];
  p->E_ext[4] = em[0][2];
  p->E_ext[5] = em[0][1];
  return GSPM_OK;
}

namespace {

struct Key {
  int64_t x, y, z;
  bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.y + 0xBF58476D1CE4E5B9ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.z + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// geometry of one tet from its four stored vertices: J = [x1-x0, x2-x0, x3-x0] (columns),
// grad phi_1..3 = rows of J^-1, grad phi_0 = -sum; returns det J
double tet_geometry(const double* x0, const double* x1, const double* x2, const double* x3,
                    double g[12]) {
  double J[3][3];
  for (int a = 0; a < 3; ++a) {
    J[a][0] = x1[a] - x0[a];
    J[a][1] = x2[a] - x0[a];
    J[a][2] = x3[a] - x0[a];
  }
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  if (!(det > 0.0)) return det;
  const double inv = 1.0 / det;
  // inverse = adjugate / det; row r of J^-1 = grad phi_{r+1}
  double Ji[3][3];
  Ji[0][0] = c00 * inv;
  Ji[1][0] = c01 * inv;
  Ji[2][0] = c02 * inv;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
  for (int a = 0; a < 3; ++a) {
    g[3 + a] = Ji[0][a];
    g[6 + a] = Ji[1][a];
    g[9 + a] = Ji[2][a];
    g[a] = -(Ji[0][a] + Ji[1][a] + Ji[2][a]);
  }
  return det;
}

// Linear hexahedron at the 2x2x2 Gauss points xi_q = s_q / sqrt(3) (weights 1): with the
// shape functions N_a = prod_d (1 + s_a,d xi_d) / 2, J_ij = dx_i / dxi_j = sum_a x_a,i dN_a/dxi_j,
// w[q] = det J_q and g[(q * 8 + a) * 3 + i] = d_i N_a = sum_j dN_a/dxi_j (J^-1)_ji.  Returns the
// smallest det J_q.
double hex_geometry(const double* const x[8], double w[8], double g[8 * 8 * 3]) {
  const double r = 1.0 / std::sqrt(3.0);
  double dmin = INFINITY;
  for (int q = 0; q < kHexGauss; ++q) {
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = r * kHexSign[q][d];
    double dN[8][3];
    for (int a = 0; a < kHexNodes; ++a)
      for (int d = 0; d < 3; ++d) {
        double v = 0.5 * kHexSign[a][d];
        for (int e = 0; e < 3; ++e)
          if (e != d) v *= 0.5 * (1.0 + kHexSign[a][e] * xi[e]);
        dN[a][d] = v;
      }
    double J[3][3] = {};
    for (int a = 0; a < kHexNodes; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] += x[a][i] * dN[a][j];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    dmin = std::min(dmin, det);
    w[q] = det;
    if (!(det > 0.0)) continue;
    const double inv = 1.0 / det;
    double Ji[3][3];  // J^-1
    Ji[0][0] = c00 * inv;
    Ji[1][0] = c01 * inv;
    Ji[2][0] = c02 * inv;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
    for (int a = 0; a < kHexNodes; ++a)
      for (int i = 0; i < 3; ++i) {
        double v = 0.0;
        for (int j = 0; j < 3; ++j) v += dN[a][j] * Ji[j][i];
        g[(q * 8 + a) * 3 + i] = v;
      }
  }
  return dmin;
}

// N_a at the Gauss points, [q][a]
struct HexN {
  double v[kHexGauss][kHexNodes];
  HexN() {
    const double r = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < kHexGauss; ++q) {
      double xi[3];
      for (int d = 0; d < 3; ++d) xi[d] = r * kHexSign[q][d];
      for (int a = 0; a < kHexNodes; ++a) v[q][a] = hex_shape(a, xi);
    }
  }
};
const HexN& hex_n() {
  static const HexN t;
  return t;
}

}  // namespace

const int kHexSign[kHexNodes][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

double hex_shape(int a, const double xi[3]) {
  return 0.125 * (1.0 + kHexSign[a][0] * xi[0]) * (1.0 + kHexSign[a][1] * xi[1]) *
         (1.0 + kHexSign[a][2] * xi[2]);
}

int64_t coarse_nodes_of(int64_t option, int64_t n) {
  return option > 0 ? option : std::max<int64_t>(512, (n + 5999) / 6000);
}

void coarse_bins(const HostMesh& hm, int64_t nodes_per_agg, int nb[3],
                 std::vector<int64_t>* bin_of) {
  const int64_t n = hm.n;
  double L[3], vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    L[a] = hm.hi[a] - hm.lo[a];
    vol *= L[a];
  }
  const double H = std::cbrt(vol * (double)std::max<int64_t>(1, nodes_per_agg) / (double)n);
  for (int a = 0; a < 3; ++a) nb[a] = (int)std::max<int64_t>(1, std::llround(L[a] / H));
  bin_of->resize(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t b[3];
    for (int a = 0; a < 3; ++a) {
      const double t = (hm.xw[3 * i + a] - hm.lo[a]) / L[a] * nb[a];
      b[a] = std::min<int64_t>(nb[a] - 1, std::max<int64_t>(0, (int64_t)std::floor(t)));
    }
    (*bin_of)[i] = b[0] + nb[0] * (b[1] + (int64_t)nb[1] * b[2]);
  }
}

int host_mesh_build(const gspm_mesh_desc* d, int ordering, int64_t coarse_nodes,
                    HostMesh* hm) {
  if (!d || !d->coords || !d->tets || d->n_nodes <= 0 || d->n_tets <= 0) {
    set_error("mesh_load: null pointer or empty mesh");
    return GSPM_EINVAL;
  }
  if (d->n_nodes > INT32_MAX) {
    set_error("mesh_load: more than 2^31-1 nodes");
    return GSPM_EINVAL;
  }
  const int64_t ns = d->n_nodes, nt = d->n_tets;
  const int nen = d->nodes_per_elem == 0 ? 4 : d->nodes_per_elem;
  if (nen != 4 && nen != kHexNodes) {
    set_error("mesh_load: nodes_per_elem %d (4: tetrahedra, 8: hexahedra)", d->nodes_per_elem);
    return GSPM_EINVAL;
  }
  const bool hex = nen == kHexNodes;
  hm->nen = nen;
  hm->n_stored = ns;
  hm->n_tets = nt;
  for (int64_t i = 0; i < 3 * ns; ++i)
    if (!std::isfinite(d->coords[i])) {
      set_error("mesh_load: non-finite coordinate at node %lld", (long long)(i / 3));
      return GSPM_EMESH;
    }
  for (int a = 0; a < 3; ++a)
    if (!(d->box_hi[a] > d->box_lo[a])) {
      set_error("mesh_load: empty box along axis %d", a);
      return GSPM_EINVAL;
    }
  for (int64_t i = 0; i < nen * nt; ++i)
    if (d->tets[i] < 0 || d->tets[i] >= ns) {
      set_error("mesh_load: element %lld references node %d outside [0, %lld)",
                (long long)(i / nen), d->tets[i], (long long)ns);
      return GSPM_EMESH;
    }
  // geometry from stored (unwrapped) coordinates
  hm->V.resize(nt);
  if (hex) {
    hm->hw.resize((int64_t)kHexGauss * nt);
    hm->hg.resize((int64_t)kHexGauss * kHexNodes * 3 * nt);
  } else {
    hm->grads.resize(12 * nt);
  }
  double min_edge = INFINITY;
  bool bad = false;
  int64_t bad_tet = -1;
#pragma omp parallel for reduction(min : min_edge)
  for (int64_t e = 0; e < nt; ++e) {
    const int32_t* t = d->tets + (int64_t)nen * e;
    const double* x[8];
    for (int k = 0; k < nen; ++k) x[k] = d->coords + 3 * (int64_t)t[k];
    double det, vol;
    if (hex) {
      double* w = &hm->hw[(int64_t)kHexGauss * e];
      det = hex_geometry(x, w, &hm->hg[(int64_t)kHexGauss * kHexNodes * 3 * e]);
      vol = 0.0;
      for (int q = 0; q < kHexGauss; ++q) vol += w[q];
    } else {
      det = tet_geometry(x[0], x[1], x[2], x[3], &hm->grads[12 * e]);
      vol = det / 6.0;
    }
    if (!(det > 0.0)) {
#pragma omp critical
      {
        if (!bad || e < bad_tet) bad_tet = e;
        bad = true;
      }
    }
    hm->V[e] = vol;
    for (int i = 0; i < nen; ++i)
      for (int j = i + 1; j < nen; ++j) {
        const double dx = x[i][0] - x[j][0], dy = x[i][1] - x[j][1], dz = x[i][2] - x[j][2];
        min_edge = std::min(min_edge, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
  }
  if (bad) {
    set_error(hex ? "mesh_load: hexahedron %lld has det(J) <= 0 at a Gauss point"
                  : "mesh_load: tet %lld has det(J) <= 0",
              (long long)bad_tet);
    return GSPM_EMESH;
  }
  // periodic wrap: hash map of quantised wrapped coordinates, ids by first occurrence
  const double tol = d->wrap_tol > 0 ? d->wrap_tol : 1e-6 * min_edge;
  hm->unique_of_stored.resize(ns);
  {
    std::unordered_map<Key, int64_t, KeyHash> table;
    table.reserve((size_t)ns);
    for (int64_t s = 0; s < ns; ++s) {
      int64_t q[3];
      for (int a = 0; a < 3; ++a) {
        double x = d->coords[3 * s + a];
        if (std::fabs(x - d->box_hi[a]) <= tol) x = d->box_lo[a];
        q[a] = (int64_t)std::floor((x - d->box_lo[a]) / tol + 0.5);
      }
      auto it = table.emplace(Key{q[0], q[1], q[2]}, (int64_t)table.size()).first;
      hm->unique_of_stored[s] = it->second;
      if (it->second == (int64_t)hm->xw.size() / 3)
        for (int a = 0; a < 3; ++a) {
          double x = d->coords[3 * s + a];
          if (std::fabs(x - d->box_hi[a]) <= tol) x = d->box_lo[a];
          hm->xw.push_back(x);
        }
    }
    hm->n = (int64_t)table.size();
    for (int a = 0; a < 3; ++a) {
      hm->lo[a] = d->box_lo[a];
      hm->hi[a] = d->box_hi[a];
    }
  }
  const int64_t n = hm->n;
  hm->tets_u.resize(nen * nt);
  hm->elem_mag.resize(nt);
  for (int64_t e = 0; e < nt; ++e) {
    int64_t* tu = &hm->tets_u[nen * e];
    for (int k = 0; k < nen; ++k) tu[k] = hm->unique_of_stored[d->tets[nen * e + k]];
    for (int k = 0; k < nen; ++k)
      for (int l = k + 1; l < nen; ++l)
        if (tu[k] == tu[l]) {
          set_error("mesh_load: element %lld collapses under the periodic wrap", (long long)e);
          return GSPM_EMESH;
        }
    hm->elem_mag[e] = d->elem_magnetic ? (d->elem_magnetic[e] ? 1 : 0) : 1;
  }
  // node flags, lumped mass, volumes
  hm->node_mag.assign(n, 0);
  hm->ML.assign(n, 0.0);
  hm->n_mag_tets = 0;
  // volumes with Neumaier-compensated sums (they normalise every volume average)
  double vs = 0.0, vc = 0.0, ms = 0.0, mc = 0.0;
  auto nsum = [](double& s, double& c, double x) {
    const double t = s + x;
    c += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  };
  const HexN& hn = hex_n();
  for (int64_t e = 0; e < nt; ++e) {
    nsum(vs, vc, hm->V[e]);
    for (int k = 0; k < nen; ++k) {
      double mk = hm->V[e] / 4.0;  // int phi_k
      if (hex) {
        mk = 0.0;
        for (int q = 0; q < kHexGauss; ++q) mk += hm->hw[kHexGauss * e + q] * hn.v[q][k];
      }
      hm->ML[hm->tets_u[nen * e + k]] += mk;
    }
    if (hm->elem_mag[e]) {
      nsum(ms, mc, hm->V[e]);
      ++hm->n_mag_tets;
      for (int k = 0; k < nen; ++k) hm->node_mag[hm->tets_u[nen * e + k]] = 1;
    }
  }
  hm->volume = vs + vc;
  hm->volume_mag = ms + mc;
  hm->n_mag_nodes = 0;
  for (int64_t i = 0; i < n; ++i) hm->n_mag_nodes += hm->node_mag[i];
  // node graph (self included), ascending columns
  std::vector<int64_t> ntp(n + 1, 0), nti(nen * nt);
  for (int64_t e = 0; e < nt; ++e)
    for (int k = 0; k < nen; ++k) ++ntp[hm->tets_u[nen * e + k] + 1];
  for (int64_t i = 0; i < n; ++i) ntp[i + 1] += ntp[i];
  {
    std::vector<int64_t> fill(ntp.begin(), ntp.end() - 1);
    for (int64_t e = 0; e < nt; ++e)
      for (int k = 0; k < nen; ++k) nti[fill[hm->tets_u[nen * e + k]]++] = e;
  }
  std::vector<std::vector<int64_t>> adj(n);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int64_t>& a = adj[i];
    for (int64_t q = ntp[i]; q < ntp[i + 1]; ++q)
      for (int k = 0; k < nen; ++k) a.push_back(hm->tets_u[nen * nti[q] + k]);
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  hm->rowptr.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) hm->rowptr[i + 1] = hm->rowptr[i] + (int64_t)adj[i].size();
  hm->cols.resize(hm->rowptr[n]);
  for (int64_t i = 0; i < n; ++i)
    std::copy(adj[i].begin(), adj[i].end(), hm->cols.begin() + hm->rowptr[i]);
  // renumbering
  hm->perm.resize(n);
  if (ordering == GSPM_ORDER_RCM) {
    std::vector<int64_t> deg(n);
    for (int64_t i = 0; i < n; ++i) deg[i] = hm->rowptr[i + 1] - hm->rowptr[i] - 1;
    auto less = [&](int64_t a, int64_t b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };
    std::vector<int64_t> by(n);
    std::iota(by.begin(), by.end(), 0);
    std::sort(by.begin(), by.end(), less);
    std::vector<uint8_t> vis(n, 0);
    std::vector<int64_t> order;
    order.reserve(n);
    std::deque<int64_t> q;
    std::vector<int64_t> nxt;
    for (int64_t st : by) {
      if (vis[st]) continue;
      vis[st] = 1;
      q.push_back(st);
      while (!q.empty()) {
        const int64_t v = q.front();
        q.pop_front();
        order.push_back(v);
        nxt.clear();
        for (int64_t p = hm->rowptr[v]; p < hm->rowptr[v + 1]; ++p) {
          const int64_t w = hm->cols[p];
          if (w != v && !vis[w]) nxt.push_back(w);
        }
        std::sort(nxt.begin(), nxt.end(), less);
        for (int64_t w : nxt) {
          vis[w] = 1;
          q.push_back(w);
        }
      }
    }
    for (int64_t i = 0; i < n; ++i) hm->perm[i] = order[n - 1 - i];
  } else if (ordering == GSPM_ORDER_NONE) {
    std::iota(hm->perm.begin(), hm->perm.end(), 0);
  } else if (ordering == GSPM_ORDER_AGGREGATE) {
    int nb[3];
    std::vector<int64_t> bin_of;
    coarse_bins(*hm, coarse_nodes_of(coarse_nodes, n), nb, &bin_of);
    std::iota(hm->perm.begin(), hm->perm.end(), 0);
    std::stable_sort(hm->perm.begin(), hm->perm.end(),
                     [&](int64_t a, int64_t b) { return bin_of[a] < bin_of[b]; });
  } else {
    set_error("mesh_load: unknown ordering %d", ordering);
    return GSPM_EINVAL;
  }
  hm->iperm.resize(n);
  for (int64_t i = 0; i < n; ++i) hm->iperm[hm->perm[i]] = i;
  return GSPM_OK;
}

void host_sell_build(const HostMesh& hm, HostSell* s) {
  const int64_t n = hm.n;
  s->n = n;
  s->nslices = (n + kSell - 1) / kSell;
  // internal-numbering rows: columns renumbered and re-sorted
  s->rp.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t o = hm.perm[i];
    s->rp[i + 1] = s->rp[i] + (hm.rowptr[o + 1] - hm.rowptr[o]);
  }
  s->ic.resize(s->rp[n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t o = hm.perm[i];
    int32_t* dst = &s->ic[s->rp[i]];
    int64_t c = 0;
    for (int64_t p = hm.rowptr[o]; p < hm.rowptr[o + 1]; ++p) dst[c++] = (int32_t)hm.iperm[hm.cols[p]];
    std::sort(dst, dst + c);
  }
  s->sptr.assign(s->nslices + 1, 0);
  s->slen.assign(s->nslices, 0);
  for (int64_t sl = 0; sl < s->nslices; ++sl) {
    int32_t mx = 0;
    for (int64_t i = sl * kSell; i < std::min(n, (sl + 1) * kSell); ++i)
      mx = std::max<int32_t>(mx, (int32_t)(s->rp[i + 1] - s->rp[i]));
    s->slen[sl] = mx;
    s->sptr[sl + 1] = s->sptr[sl] + (int64_t)mx * kSell;
  }
  s->entries = s->sptr[s->nslices];
  s->col.assign(s->entries, 0);
#pragma omp parallel for schedule(static)
  for (int64_t sl = 0; sl < s->nslices; ++sl) {
    for (int lane = 0; lane < kSell; ++lane) {
      const int64_t i = sl * kSell + lane;
      const int64_t len = i < n ? s->rp[i + 1] - s->rp[i] : 0;
      for (int32_t k = 0; k < s->slen[sl]; ++k)
        s->col[s->sptr[sl] + (int64_t)k * kSell + lane] =
            k < len ? s->ic[s->rp[i] + k] : (int32_t)(i < n ? i : 0);
    }
  }
}

void host_assemble(const HostMesh& hm, const HostSell& s, const Params& p, HostOps* ops) {
  const int64_t n = hm.n, E = s.entries;
  ops->Kms.assign(E, 0.0);
  ops->Aeps.assign(E, 0.0);
  ops->Aaeps.assign(E, 0.0);
  ops->M.assign(E, 0.0);
  ops->F.assign(3 * E, 0.0);
  ops->G.assign(3 * E, 0.0);
  ops->Kmech.assign(9 * E, 0.0);
  ops->Agg.assign(E, 0.0);
  ops->AggT.assign(E, 0.0);
  ops->ML.assign(n, 0.0);
  ops->w.assign(n, 0.0);
  ops->invML.assign(n, 0.0);
  ops->mag.assign(n, 0);
  ops->pin = hm.iperm[0];
  // node -> incident elements, ascending element index
  const int nen = hm.nen;
  const bool hex = nen == kHexNodes;
  const HexN& hn = hex_n();
  std::vector<int64_t> ntp(n + 1, 0), nti(nen * hm.n_tets);
  for (int64_t e = 0; e < hm.n_tets; ++e)
    for (int k = 0; k < nen; ++k) ++ntp[hm.tets_u[nen * e + k] + 1];
  for (int64_t i = 0; i < n; ++i) ntp[i + 1] += ntp[i];
  {
    std::vector<int64_t> fill(ntp.begin(), ntp.end() - 1);
    for (int64_t e = 0; e < hm.n_tets; ++e)
      for (int k = 0; k < nen; ++k) nti[fill[hm.tets_u[nen * e + k]]++] = e;
  }
  std::vector<double> vsum(n, 0.0);  // sum of the volumes of the elements at each row
  const double C11 = p.C11, C12 = p.C12, C44 = p.C44, eps = p.eps, aeps = p.alpha * p.eps;
#pragma omp parallel
  {
    std::vector<double> kms, km, mm, f, g, k9, bb;
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t o = hm.perm[i];
      const int32_t* rc = &s.ic[s.rp[i]];
      const int len = (int)(s.rp[i + 1] - s.rp[i]);
      kms.assign(len, 0.0); km.assign(len, 0.0); mm.assign(len, 0.0);
      f.assign(3 * len, 0.0); g.assign(3 * len, 0.0); k9.assign(9 * len, 0.0);
      bb.assign(len, 0.0);
      double ml = 0.0, vs = 0.0;
      // K_ab = sum_cd gk_c C_acbd gl_d; in the cube axes
      // K_ab = d_ab [(C11 - C44) gk_a gl_a + C44 gk.gl] + (1 - d_ab)[C12 gk_a gl_b + C44 gk_b gl_a]
      auto kmech_add = [&](double* k9p, double wq, const double* gk, const double* gl) {
        const double dot = gk[0] * gl[0] + gk[1] * gl[1] + gk[2] * gl[2];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            double v;
            if (p.rotated) {
              v = 0.0;
              for (int c = 0; c < 3; ++c)
                for (int dd = 0; dd < 3; ++dd)
                  v += gk[c] * p.Cm[((a * 3 + c) * 3 + b) * 3 + dd] * gl[dd];
            } else {
              v = a == b ? (C11 - C44) * gk[a] * gl[a] + C44 * dot
                         : C12 * gk[a] * gl[b] + C44 * gk[b] * gl[a];
            }
            k9p[3 * a + b] += wq * v;
          }
      };
      for (int64_t q = ntp[o]; q < ntp[o + 1]; ++q) {
        const int64_t e = nti[q];
        const int64_t* t = &hm.tets_u[nen * e];
        int k = 0;
        while (t[k] != o) ++k;
        const double V = hm.V[e];
        const bool me = hm.elem_mag[e] != 0;
        vs += V;
        if (!hex) {
          // linear tetrahedron: every integral in closed form
          const double* gk = &hm.grads[12 * e + 3 * k];
          ml += V / 4.0;
          for (int l = 0; l < 4; ++l) {
            const int32_t j = (int32_t)hm.iperm[t[l]];
            int pos = 0;
            while (rc[pos] != j) ++pos;
            const double* gl = &hm.grads[12 * e + 3 * l];
            const double dot = gk[0] * gl[0] + gk[1] * gl[1] + gk[2] * gl[2];
            kms[pos] += V * dot;
            bb[pos] += V / 4.0;  // B_ij = sum_{e containing i, j} V_e / (nodes per element)
            if (me) {
              km[pos] += V * dot;
              mm[pos] += V * (k == l ? 2.0 : 1.0) / 20.0;
            }
            for (int a = 0; a < 3; ++a) {
              f[3 * pos + a] += -(V / 4.0) * gl[a];   // -int phi_i d_a phi_j
              g[3 * pos + a] += (V / 4.0) * gk[a];    //  int phi_j d_a phi_i
            }
            kmech_add(&k9[9 * pos], V, gk, gl);
          }
        } else {
          // trilinear hexahedron: the same integrals by 2x2x2 Gauss quadrature
          const double* w = &hm.hw[(int64_t)kHexGauss * e];
          const double* hg = &hm.hg[(int64_t)kHexGauss * kHexNodes * 3 * e];
          for (int qq = 0; qq < kHexGauss; ++qq) ml += w[qq] * hn.v[qq][k];
          for (int l = 0; l < kHexNodes; ++l) {
            const int32_t j = (int32_t)hm.iperm[t[l]];
            int pos = 0;
            while (rc[pos] != j) ++pos;
            bb[pos] += V / kHexNodes;
            for (int qq = 0; qq < kHexGauss; ++qq) {
              const double wq = w[qq], Nk = hn.v[qq][k], Nl = hn.v[qq][l];
              const double* gk = hg + (qq * 8 + k) * 3;
              const double* gl = hg + (qq * 8 + l) * 3;
              const double dot = gk[0] * gl[0] + gk[1] * gl[1] + gk[2] * gl[2];
              kms[pos] += wq * dot;
              if (me) {
                km[pos] += wq * dot;
                mm[pos] += wq * Nk * Nl;
              }
              for (int a = 0; a < 3; ++a) {
                f[3 * pos + a] += -wq * Nk * gl[a];
                g[3 * pos + a] += wq * Nl * gk[a];
              }
              kmech_add(&k9[9 * pos], wq, gk, gl);
            }
          }
        }
      }
      const int64_t sl = i / kSell, lane = i % kSell;
      for (int pos = 0; pos < len; ++pos) {
        const int64_t ent = s.sptr[sl] + (int64_t)pos * kSell + lane;
        const int64_t vb = ent - lane;  // value base for B-valued matrices
        ops->Kms[ent] = kms[pos];
        ops->M[ent] = mm[pos];
        ops->Aeps[ent] = mm[pos] + eps * km[pos];
        ops->Aaeps[ent] = mm[pos] + aeps * km[pos];
        for (int a = 0; a < 3; ++a) {
          ops->F[vb * 3 + a * kSell + lane] = f[3 * pos + a];
          ops->G[vb * 3 + a * kSell + lane] = g[3 * pos + a];
        }
        for (int b = 0; b < 9; ++b) ops->Kmech[vb * 9 + b * kSell + lane] = k9[9 * pos + b];
      }
      // element-message average: A_ij = B_ij / (sum of the volumes of the elements at i)
      for (int pos = 0; pos < len; ++pos)
        ops->Agg[s.sptr[sl] + (int64_t)pos * kSell + lane] = bb[pos] / vs;
      vsum[i] = vs;
      ops->ML[i] = ml;
      ops->w[i] = ml / hm.volume;
      ops->invML[i] = 1.0 / ml;
      ops->mag[i] = hm.node_mag[o];
      if (!hm.node_mag[o]) {  // rows off Omega_m: identity in the GSPM operators
        for (int pos = 0; pos < len; ++pos)
          if (rc[pos] == i) {
            const int64_t ent = s.sptr[sl] + (int64_t)pos * kSell + lane;
            ops->Aeps[ent] = ops->Aaeps[ent] = 1.0;
          }
      }
    }
  }
  // A^T at (i, j) = A_ji = B_ij / vsum_j  (B is symmetric)
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t sl = i / kSell, lane = i % kSell;
    const int len = (int)(s.rp[i + 1] - s.rp[i]);
    for (int pos = 0; pos < len; ++pos) {
      const int64_t ent = s.sptr[sl] + (int64_t)pos * kSell + lane;
      const int32_t j = s.ic[s.rp[i] + pos];
      ops->AggT[ent] = ops->Agg[ent] * vsum[i] / vsum[j];
    }
  }
}

void host_batch_build(std::vector<HostMesh>& hm, std::vector<HostSell>& hs,
                      std::vector<HostOps>& ops, HostBatch* b) {
  const int S = (int)hm.size();
  b->seg_row0.resize(S);
  b->seg_nrow.resize(S);
  b->seg_pin.resize(S);
  b->seg_sl0.resize(S);
  b->seg_nsl.resize(S);
  b->seg_node0.resize(S);
  b->seg_nmag.resize(S);
  b->seg_h.resize(S);
  int64_t sl = 0, node = 0, entries = 0;
  for (int s = 0; s < S; ++s) {
    b->seg_sl0[s] = sl;
    b->seg_nsl[s] = hs[s].nslices;
    b->seg_row0[s] = sl * kSell;
    b->seg_nrow[s] = hm[s].n;
    b->seg_pin[s] = b->seg_row0[s] + ops[s].pin;
    b->seg_node0[s] = node;
    b->seg_nmag[s] = hm[s].n_mag_nodes;
    b->seg_h[s] = std::cbrt(hm[s].volume / (double)hm[s].n);
    sl += hs[s].nslices;
    node += hm[s].n;
    entries += hs[s].entries;
  }
  b->n_nodes = node;
  b->n_mag_nodes = 0;
  for (int s = 0; s < S; ++s) b->n_mag_nodes += hm[s].n_mag_nodes;
  b->seg_of_slice.resize(sl);
  for (int s = 0; s < S; ++s)
    for (int64_t k = 0; k < hs[s].nslices; ++k) b->seg_of_slice[b->seg_sl0[s] + k] = s;
  if (S == 1) {  // no copies for a single mesh
    b->sell = std::move(hs[0]);
    b->ops = std::move(ops[0]);
    b->perm = hm[0].perm;
    return;
  }
  const int64_t rows = b->seg_row0[S - 1] + hm[S - 1].n;
  HostSell& c = b->sell;
  c.n = rows;
  c.nslices = sl;
  c.entries = entries;
  c.sptr.assign(sl + 1, 0);
  c.slen.assign(sl, 0);
  c.col.assign(entries, 0);
  HostOps& o = b->ops;
  o.Kms.resize(entries); o.Aeps.resize(entries); o.Aaeps.resize(entries); o.M.resize(entries);
  o.Agg.resize(entries); o.AggT.resize(entries);
  o.F.resize(3 * entries); o.G.resize(3 * entries); o.Kmech.resize(9 * entries);
  o.ML.assign(rows, 1.0); o.w.assign(rows, 0.0); o.invML.assign(rows, 0.0);
  o.mag.assign(rows, 0);
  b->perm.assign(rows, -1);
  int64_t e0 = 0;
  for (int s = 0; s < S; ++s) {
    const HostSell& h = hs[s];
    const int64_t r0 = b->seg_row0[s], s0 = b->seg_sl0[s];
    for (int64_t k = 0; k < h.nslices; ++k) {
      c.sptr[s0 + k] = e0 + h.sptr[k];
      c.slen[s0 + k] = h.slen[k];
    }
    for (int64_t e = 0; e < h.entries; ++e) c.col[e0 + e] = (int32_t)(h.col[e] + r0);
    auto cp = [&](std::vector<double>& dst, const std::vector<double>& src, int64_t B) {
      std::copy(src.begin(), src.end(), dst.begin() + e0 * B);
    };
    cp(o.Kms, ops[s].Kms, 1); cp(o.Aeps, ops[s].Aeps, 1); cp(o.Aaeps, ops[s].Aaeps, 1);
    cp(o.M, ops[s].M, 1); cp(o.Agg, ops[s].Agg, 1); cp(o.AggT, ops[s].AggT, 1);
    cp(o.F, ops[s].F, 3); cp(o.G, ops[s].G, 3); cp(o.Kmech, ops[s].Kmech, 9);
    for (int64_t i = 0; i < hm[s].n; ++i) {
      o.ML[r0 + i] = ops[s].ML[i];
      o.w[r0 + i] = ops[s].w[i];
      o.invML[r0 + i] = ops[s].invML[i];
      o.mag[r0 + i] = ops[s].mag[i];
      b->perm[r0 + i] = b->seg_node0[s] + hm[s].perm[i];
    }
    e0 += h.entries;
    // release the per-mesh copies as we go
    ops[s] = HostOps();
    hs[s].col.clear();
    hs[s].col.shrink_to_fit();
  }
  c.sptr[sl] = e0;
}

}  // namespace gspm

namespace gspm {

// sum_{k < len} a[k] b[k] with four independent partial sums (the dependent chain of a single
// sum bounds the host's dense factorisation)
static inline double dot4(const double* a, const double* b, int64_t len) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t k = 0;
  for (; k + 4 <= len; k += 4) {
    s0 += a[k] * b[k];
    s1 += a[k + 1] * b[k + 1];
    s2 += a[k + 2] * b[k + 2];
    s3 += a[k + 3] * b[k + 3];
  }
  for (; k < len; ++k) s0 += a[k] * b[k];
  return (s0 + s1) + (s2 + s3);
}

// acc[x][y] += sum_t a[x][t] b[y][t] for t < len: a 4 x 4 register tile of dot products of
// rows, each loaded value serving four products, two consecutive t per vector lane pair (GCC
// vector extension: SSE2 or NEON, the same pairwise order on either), odd tail in order
typedef double Dbl2 __attribute__((vector_size(16)));
static inline Dbl2 load2(const double* p) {
  Dbl2 v;
  std::memcpy(&v, p, sizeof(v));
  return v;
}
static inline void tile4x4(const double* const a[4], const double* const b[4], int64_t len,
                           double (&acc)[4][4]) {
  Dbl2 s[4][4];
  for (int x = 0; x < 4; ++x)
    for (int y = 0; y < 4; ++y) s[x][y] = Dbl2{0.0, 0.0};
  int64_t t = 0;
  for (; t + 2 <= len; t += 2) {
    const Dbl2 a0 = load2(a[0] + t), a1 = load2(a[1] + t), a2 = load2(a[2] + t),
               a3 = load2(a[3] + t);
    const Dbl2 b0 = load2(b[0] + t), b1 = load2(b[1] + t), b2 = load2(b[2] + t),
               b3 = load2(b[3] + t);
    s[0][0] += a0 * b0; s[0][1] += a0 * b1; s[0][2] += a0 * b2; s[0][3] += a0 * b3;
    s[1][0] += a1 * b0; s[1][1] += a1 * b1; s[1][2] += a1 * b2; s[1][3] += a1 * b3;
    s[2][0] += a2 * b0; s[2][1] += a2 * b1; s[2][2] += a2 * b2; s[2][3] += a2 * b3;
    s[3][0] += a3 * b0; s[3][1] += a3 * b1; s[3][2] += a3 * b2; s[3][3] += a3 * b3;
  }
  for (int x = 0; x < 4; ++x)
    for (int y = 0; y < 4; ++y) acc[x][y] += s[x][y][0] + s[x][y][1];
  for (; t < len; ++t)
    for (int x = 0; x < 4; ++x)
      for (int y = 0; y < 4; ++y) acc[x][y] += a[x][t] * b[y][t];
}

// Blocked right-looking Cholesky of the SPD matrix A (n x n, row-major, lower factor in place):
// per block of kb columns, the diagonal block unblocked, the rows below it by forward
// substitution, then the trailing lower triangle updated by the block's rank-kb product in
// 4 x 4 tiles.
static bool chol_blocked(std::vector<double>& A, int64_t n) {
  constexpr int64_t NB = 128;
  for (int64_t k = 0; k < n; k += NB) {
    const int64_t kb = std::min(NB, n - k);
    for (int64_t j = k; j < k + kb; ++j) {
      const double d = A[j * n + j] - dot4(&A[j * n + k], &A[j * n + k], j - k);
      if (!(d > 0.0)) return false;
      const double ljj = std::sqrt(d);
      A[j * n + j] = ljj;
      for (int64_t i = j + 1; i < k + kb; ++i)
        A[i * n + j] = (A[i * n + j] - dot4(&A[i * n + k], &A[j * n + k], j - k)) / ljj;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = k + kb; i < n; ++i)
      for (int64_t j = k; j < k + kb; ++j)
        A[i * n + j] = (A[i * n + j] - dot4(&A[i * n + k], &A[j * n + k], j - k)) / A[j * n + j];
    const int64_t m0 = k + kb, nt = (n - m0 + 3) / 4;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t bi = 0; bi < nt; ++bi) {
      const int64_t i0 = m0 + 4 * bi;
      for (int64_t j0 = m0; j0 <= i0; j0 += 4) {
        double acc[4][4] = {};
        const double* a[4];
        const double* b[4];
        for (int x = 0; x < 4; ++x) {
          a[x] = &A[std::min(i0 + x, n - 1) * n + k];
          b[x] = &A[std::min(j0 + x, n - 1) * n + k];
        }
        tile4x4(a, b, kb, acc);
        for (int x = 0; x < 4; ++x)
          for (int y = 0; y < 4; ++y) {
            const int64_t i = i0 + x, j = j0 + y;
            if (i < n && j <= i) A[i * n + j] -= acc[x][y];
          }
      }
    }
  }
  return true;
}

// Explicit inverse of the SPD matrix A (overwritten by its Cholesky factor L); false if a pivot
// is not positive.  W = L^-1 is formed transposed (Wt row j = column j of W, zero left of the
// diagonal) four rows at a time: Wt[j][i] = (delta_ij - sum_{k<i} L[i][k] Wt[j][k]) / L[i][i],
// the part k < i0 of each 4 x 4 block of (j, i) as a register tile, the rest in order.  Then
// A^-1 = W^T W: entry (a, b >= a) = sum_k Wt[a][k] Wt[b][k], again in 4 x 4 tiles, and the lower
// triangle mirrored.
static bool spd_inverse(std::vector<double>& A, int64_t n, std::vector<double>* inv) {
  if (!chol_blocked(A, n)) return false;
  std::vector<double> Wt(n * n, 0.0);
  const int64_t nb = (n + 3) / 4;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t bj = 0; bj < nb; ++bj) {
    const int64_t j0 = 4 * bj;
    for (int64_t i0 = j0; i0 < n; i0 += 4) {
      double acc[4][4] = {};  // [x: row j0 + x of Wt][y: column i0 + y]
      const double* a[4];
      const double* b[4];
      for (int x = 0; x < 4; ++x) {
        a[x] = &Wt[std::min(j0 + x, n - 1) * n + j0];
        b[x] = &A[std::min(i0 + x, n - 1) * n + j0];
      }
      tile4x4(a, b, i0 - j0, acc);
      for (int y = 0; y < 4 && i0 + y < n; ++y) {
        const int64_t i = i0 + y;
        for (int x = 0; x < 4 && j0 + x < n; ++x) {
          const int64_t j = j0 + x;
          if (i < j) continue;
          double s = acc[x][y];
          for (int64_t k = i0; k < i; ++k) s += A[i * n + k] * Wt[j * n + k];
          Wt[j * n + i] = ((i == j ? 1.0 : 0.0) - s) / A[i * n + i];
        }
      }
    }
  }
  inv->assign(n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ba = 0; ba < nb; ++ba) {
    const int64_t a0 = 4 * ba;
    for (int64_t b0 = a0; b0 < n; b0 += 4) {
      double acc[4][4] = {};
      const double* a[4];
      const double* b[4];
      for (int x = 0; x < 4; ++x) {
        a[x] = &Wt[std::min(a0 + x, n - 1) * n + b0];
        b[x] = &Wt[std::min(b0 + x, n - 1) * n + b0];
      }
      tile4x4(a, b, n - b0, acc);
      for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
          const int64_t r = a0 + x, c = b0 + y;
          if (r < n && c < n && c >= r) (*inv)[r * n + c] = acc[x][y];
        }
    }
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < i; ++c) (*inv)[i * n + c] = (*inv)[c * n + i];
  return true;
}

double bf16_round(double v) {
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  float r;
  std::memcpy(&r, &u, sizeof(r));
  return (double)r;
}

int coarse_round_spd(const double* A, int64_t n, int bf16, std::vector<double>* stored,
                     double* shift) {
  stored->assign(n * n, 0.0);
  *shift = 0.0;
  double dmax = 0.0;
  for (int64_t i = 0; i < n; ++i) dmax = std::max(dmax, std::fabs(A[i * n + i]));
  std::vector<double> work;
  // shifts 0, 2^-8 dmax, ..., dmax: a shift beyond max_i S_ii no longer repairs rounding
  for (int attempt = 0; attempt <= 9; ++attempt) {
    const double sh = *shift;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        const double v = 0.5 * (A[i * n + j] + A[j * n + i]) + (i == j ? sh : 0.0);
        (*stored)[i * n + j] = bf16 ? bf16_round(v) : v;
      }
    if (!bf16 && attempt == 0) return GSPM_OK;  // FP64 storage: the symmetric part itself
    work = *stored;
    if (n == 0 || chol_blocked(work, n)) return GSPM_OK;
    *shift = sh > 0.0 ? 2.0 * sh : std::ldexp(dmax, -8);
  }
  set_error("coarse inverse: not positive definite after rounding with any diagonal shift up to "
            "its largest diagonal entry");
  return GSPM_EMESH;
}

int host_coarse_build(const HostMesh& hm, const HostSell& s, const HostOps& ops,
                      int64_t nodes_per_agg, int bf16, HostCoarse* c) {
  const int64_t n = hm.n;
  std::vector<int64_t> bin_of;
  coarse_bins(hm, nodes_per_agg, c->nb, &bin_of);
  const int64_t nbins = (int64_t)c->nb[0] * c->nb[1] * c->nb[2];
  std::vector<int64_t> id(nbins, -1);
  for (int64_t i = 0; i < n; ++i) id[bin_of[i]] = 0;
  int64_t na = 0;
  for (int64_t b = 0; b < nbins; ++b)
    if (id[b] == 0) id[b] = na++;
  c->n_agg = na;
  c->agg.resize(n);
  for (int64_t i = 0; i < n; ++i) c->agg[i] = (int32_t)id[bin_of[hm.perm[i]]];
  // P^T K P and the inverse diagonals from the assembled SELL values (internal numbering)
  const int64_t n3 = 3 * na;
  c->Kc_mech.assign(n3 * n3, 0.0);
  c->Kc_ms.assign(na * na, 0.0);
  c->dinv_mech.assign(3 * n, 0.0);
  c->dinv_ms.assign(n, 0.0);
  constexpr int64_t kSell = 32;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t sl = i / kSell, lane = i % kSell, I = c->agg[i];
    const int len = (int)(s.rp[i + 1] - s.rp[i]);
    for (int pos = 0; pos < len; ++pos) {
      const int64_t j = s.ic[s.rp[i] + pos], J = c->agg[j];
      const int64_t ent = s.sptr[sl] + (int64_t)pos * kSell + lane, vb = ent - lane;
      c->Kc_ms[I * na + J] += ops.Kms[ent];
      if (j == i) c->dinv_ms[i] = 1.0 / ops.Kms[ent];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const double v = ops.Kmech[vb * 9 + (3 * a + b) * kSell + lane];
          c->Kc_mech[(3 * I + a) * n3 + 3 * J + b] += v;
          if (j == i && a == b) c->dinv_mech[3 * i + a] = 1.0 / v;
        }
    }
  }
  // regularise on the constants of each component and invert
  auto regularised_inverse = [&](const std::vector<double>& K, int64_t nc, int comps,
                                 std::vector<double>* inv) -> bool {
    std::vector<double> A(K);
    double tr = 0.0;
    for (int64_t i = 0; i < nc; ++i) tr += A[i * nc + i];
    if (!(tr > 0.0) || nc == comps) {
      // one aggregate: P^T K P = 0 (constants only), no coarse correction
      inv->assign(nc * nc, 0.0);
      return true;
    }
    const double rho = tr / (double)nc / (double)(nc / comps);
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t j = 0; j < nc; ++j)
        if (i % comps == j % comps) A[i * nc + j] += rho;
    return spd_inverse(A, nc, inv);
  };
  if (!regularised_inverse(c->Kc_mech, n3, 3, &c->inv_mech) ||
      !regularised_inverse(c->Kc_ms, na, 1, &c->inv_ms)) {
    set_error("mesh_load: coarse operator of the preconditioner is not positive definite");
    return GSPM_EMESH;
  }
  // the device's copies: checked positive definite after rounding (one aggregate: no coarse
  // correction, the inverse is all zero and stays so)
  if (na > 1) {
    const int st1 = coarse_round_spd(c->inv_mech.data(), n3, bf16, &c->store_mech, &c->shift_mech);
    if (st1 != GSPM_OK) return st1;
    const int st2 = coarse_round_spd(c->inv_ms.data(), na, bf16, &c->store_ms, &c->shift_ms);
    if (st2 != GSPM_OK) return st2;
  } else {
    c->store_mech = c->inv_mech;
    c->store_ms = c->inv_ms;
  }
  return GSPM_OK;
}

}  // namespace gspm
