// Internal declarations of the GSPM library (host mesh layer, kernel launchers, context).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gspm.h"

namespace gspm {

constexpr int kSell = 32;  // SELL slice height = warp width: one thread per row, warp per slice

void set_error(const char* fmt, ...);

// Dimensionless constants of App. B and the material laws (SI inputs reduced once).
struct Params {
  double Ms, mu0, gamma0, l_d;
  double scale;     // mu0 Ms^2
  double A_star;    // 2A / (mu0 Ms^2 l_d^2)
  double kappa;     // 2 K1 / (mu0 Ms^2)
  double dtau;      // gamma0 Ms dt
  double alpha;
  double eps;       // A* dtau
  double C11, C12, C44;
  double l100, l111;
  double me_coef;   // 3 / (mu0 Ms^2)
  double Nd[9];
  double E_ext[6];  // C^-1 sigma_ext, Voigt order, tensor shear components
  // App. D: v_mesh = R v_crystal; rotated = R is not the identity.  Cm = the stiffness tensor
  // C_ijkl in the mesh axes (index (((i*3 + j)*3 + k)*3 + l)), used for K^mech when rotated.
  double R[9];
  int rotated;
  double Cm[81];
};
int make_params(const gspm_material* mat, const gspm_options* opt, Params* p);

// Host-side mesh after validation, periodic wrap and (optional) renumbering.
// Linear hexahedra: 2x2x2 Gauss points, reference corner signs and shape-function values
constexpr int kHexNodes = 8, kHexGauss = 8;
extern const int kHexSign[kHexNodes][3];
double hex_shape(int a, const double xi[3]);  // N_a(xi)

struct HostMesh {
  int64_t n_stored = 0, n_tets = 0, n = 0;  // n = unique nodes; n_tets = elements
  int nen = 4;                               // nodes per element: 4 tetrahedra, 8 hexahedra
  std::vector<int64_t> unique_of_stored;     // [n_stored]
  std::vector<int64_t> tets_u;               // [n_tets*nen] unique (original) node ids
  std::vector<uint8_t> elem_mag;             // [n_tets]
  std::vector<double> V;                     // [n_tets]
  std::vector<double> grads;                 // tetrahedra: [n_tets*12], (k*3 + a) = d_a phi_k
  std::vector<double> hw;                    // hexahedra: [n_tets*8] det J x weight per Gauss point
  std::vector<double> hg;                    // hexahedra: [n_tets*8*8*3] (q, k, a) = d_a phi_k at q
  std::vector<uint8_t> node_mag;             // [n] original numbering
  std::vector<int64_t> rowptr, cols;         // node graph, original numbering, ascending
  std::vector<int64_t> perm, iperm;          // perm[internal] = original, iperm = inverse
  std::vector<double> ML;                    // lumped mass, original numbering
  std::vector<double> xw;                    // [3n] wrapped coordinates (first stored copy)
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // periodic box
  double volume = 0, volume_mag = 0;
  int64_t n_mag_nodes = 0, n_mag_tets = 0;
};
// coarse_nodes: the option of that name (GSPM_ORDER_AGGREGATE groups the rows by the
// aggregates of coarse_nodes_of(coarse_nodes, n) nodes)
int host_mesh_build(const gspm_mesh_desc* d, int ordering, int64_t coarse_nodes, HostMesh* hm);

// Aggregate size: the option when positive, else max(512, n / 6000)
int64_t coarse_nodes_of(int64_t option, int64_t n);
// Coordinate bins of about nodes_per_agg nodes: edge H = (V nodes_per_agg / n)^(1/3), nb[a] =
// round(L_a / H) bins per axis; bin_of[i] (x fastest) for every unique node i, from its
// wrapped coordinates.
void coarse_bins(const HostMesh& hm, int64_t nodes_per_agg, int nb[3],
                 std::vector<int64_t>* bin_of);

// SELL-32 layout of the node graph in internal numbering.  Entry e of row i (k-th column of
// the row, ascending) sits at sptr[i/32] + k*32 + i%32.  A matrix with B values per entry stores
// value b of entry e at (e - lane)*B + b*32 + lane (lane = i%32): all 32 rows of a slice read one
// contiguous 32-value run per (k, b).
struct HostSell {
  int64_t n = 0, nslices = 0, entries = 0;
  std::vector<int64_t> sptr;   // [nslices+1]
  std::vector<int32_t> slen;   // [nslices]
  std::vector<int32_t> col;    // [entries], padding points at the row itself
  std::vector<int64_t> rp;     // internal-numbering row pointer into ic (unpadded)
  std::vector<int32_t> ic;     // internal-numbering ascending columns
};
void host_sell_build(const HostMesh& hm, HostSell* s);

// Assembled operators, double, SELL layout, internal numbering.
struct HostOps {
  std::vector<double> Kms, Aeps, Aaeps, M;  // scalar (B = 1)
  std::vector<double> F, G;                 // B = 3: F_{ij,a} = -int phi_i d_a phi_j,
                                            //        G_{ij,a} =  int phi_j d_a phi_i
  std::vector<double> Kmech;                // B = 9, row-major 3x3 block (a*3 + b)
  std::vector<double> Agg, AggT;            // B = 1: element-message averaging A and A^T
  std::vector<double> ML, w, invML;         // internal numbering; w = M_L / V
  std::vector<uint8_t> mag;                 // internal numbering
  int64_t pin = 0;                          // internal index of unique node 0
};
void host_assemble(const HostMesh& hm, const HostSell& s, const Params& p, HostOps* ops);

// Two-level preconditioner of the K^ms and K^mech solves: plain aggregation P (node i -> its
// aggregate, the same for every displacement component), coarse operators P^T K P, their
// inverses after the null space (the constants of each component) is shifted by
// rho / n_agg * 1 1^T, and the inverse diagonals of K (the fine-level Jacobi part).
// Aggregates: the periodic box cut into about n / nodes_per_agg equal bins, empty bins
// dropped, ids in bin order.
struct HostCoarse {
  int64_t n_agg = 0;
  int nb[3] = {1, 1, 1};               // bins per axis
  std::vector<int32_t> agg;            // [n] aggregate of each internal row
  std::vector<double> Kc_mech, Kc_ms;  // [3 n_agg]^2, [n_agg]^2 row-major, unregularised
  std::vector<double> inv_mech, inv_ms;
  std::vector<double> dinv_mech, dinv_ms;  // [3 n], [n]
  // the inverses as the device stores them (coarse_round_spd), widened to FP64, and the
  // diagonal shift that made the rounded matrix positive definite (0 when it already was)
  std::vector<double> store_mech, store_ms;
  double shift_mech = 0.0, shift_ms = 0.0;
};
// bf16: the device keeps the coarse inverses in bfloat16 (mixed precision), else in FP64
int host_coarse_build(const HostMesh& hm, const HostSell& s, const HostOps& ops,
                      int64_t nodes_per_agg, int bf16, HostCoarse* c);

// Storage of a dense symmetric positive definite matrix (the coarse inverse): its symmetric part
// S = (A + A^T) / 2, rounded entry by entry to bfloat16 (round to nearest even of the FP32 value)
// when bf16, else kept in FP64.  The rounded matrix (widened to FP64) must pass a Cholesky
// factorisation; if it does not, a diagonal shift s is added before rounding, s = 2^-8 max_i
// S_ii and doubled until it does.  Returns GSPM_OK with `stored` [n*n] and `shift`, or
// GSPM_EMESH if no shift up to max_i S_ii succeeds (A is not positive definite).
int coarse_round_spd(const double* A, int64_t n, int bf16, std::vector<double>* stored,
                     double* shift);
double bf16_round(double v);  // the value of v rounded to bfloat16 (nearest even), as FP64

// A batch of meshes ("segments") concatenated slice-aligned: segment s owns the rows
// [seg_row0[s], seg_row0[s] + seg_nrow[s]) (its last slice padded with empty rows when another
// segment follows) and the ABI nodes [seg_node0[s], seg_node0[s] + seg_nrow[s]).
struct HostBatch {
  HostSell sell;                       // combined node graph (n = all rows incl. padding)
  HostOps ops;                         // combined values and per-row arrays
  std::vector<int64_t> perm;           // [rows] ABI node of each row, -1 for padding
  std::vector<int32_t> seg_of_slice;   // [nslices]
  std::vector<int64_t> seg_row0, seg_nrow, seg_pin, seg_sl0, seg_nsl, seg_node0, seg_nmag;
  std::vector<double> seg_h;           // node spacing (V / n)^(1/3)
  std::vector<HostCoarse> coarse;      // per segment (empty without the preconditioner)
  int64_t n_nodes = 0;                 // ABI nodes of the batch
  int64_t n_mag_nodes = 0;
};
// Consumes (moves from) the per-mesh pieces.
void host_batch_build(std::vector<HostMesh>& hm, std::vector<HostSell>& hs,
                      std::vector<HostOps>& ops, HostBatch* b);

}  // namespace gspm
