// Host-side set-up of a spectral-element problem: GLL tables, numbering,
// patch tables, pencil eigen-tables, coarse Q1 matrix and its AMG hierarchy.
// Everything here runs once per handle (or per mask change), on the CPU, in
// FP64. The device side only receives the finished tables.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace sem {

// VTK hex corner c has reference bits (xi, eta, zeta) = kCornerBits[c].
extern const int kCornerBits[8][3];
int corner_of_bits(int a, int b, int c);

// GLL points t_0..t_n on [-1, 1] and weights rho_i (Sec. 2.1, Sec. 2.4).
void gll(int n, std::vector<double>& t, std::vector<double>& rho);
// Dhat[i*(n+1) + m] = phi_m'(t_i) (Eq. D, used as d/dxi at node i).
std::vector<double> derivative_matrix(int n, const std::vector<double>& t);

struct Csr {
  int n = 0, m = 0;                  // rows, columns
  std::vector<int> ptr, col;         // sorted column indices per row
  std::vector<double> val;
};

// Result of numbering a mesh (Sec. 2.2): elements in the library's order.
struct Numbering {
  int n = 0, p = 0;
  int64_t ne = 0, nv = 0, G = 0;
  int64_t Gi = 0;                    // DOFs 0..Gi-1: element interiors, e (n-1)^3 + local order
  std::vector<int64_t> elem_perm;    // library element e -> input element elem_perm[e]
  std::vector<int> hexv;             // [ne][8] input vertex ids, library element order
  std::vector<int> l2g;              // [ne * p^3], local node i + p(j + p k)
  std::vector<uint8_t> boundary;     // [G] 1 = on a boundary face
  std::vector<int> vert_dof;         // [nv] global DOF of each input vertex
  std::vector<int> face_elem;        // [ne][6] neighbour element across each face, -1 if none
  std::vector<int> face_idx;         // [ne][6] that neighbour's face index
};

// Builds the numbering; returns "" or an error message (non-manifold mesh).
std::string number_mesh(const double* xyz, int64_t nv, const int64_t* hex, int64_t ne, int n,
                        Numbering& out);

// g2l CSR over local nodes (ascending local index per DOF), owner = first local copy.
void gather_csr(const Numbering& nb, std::vector<int>& off, std::vector<int>& idx,
                std::vector<int>& owner);

// Extended-box patch table (Sec. 4.2): ip[e][(I+1) + P((J+1) + P(K+1))] = global DOF of
// box node (I, J, K), -1 <= I,J,K <= n+1, or -1 if absent. Face layers only, or (full)
// also the edge and corner layers: the (n+3)^3 nodes per subdomain that Sec. 4.2 counts.
std::vector<int> patch_table(const Numbering& nb, bool full = false);

// Extended 1D pencil (rows -1..n+1) stiffness K and diagonal mass M, and the
// generalised eigenpairs K S = M S diag(ev), S^T M S = I; S[row*P + mode]. The first
// ceil(P/2) modes are exactly even under the reflection row -> P-1-row, the rest odd.
void pencil_tables(int n, const std::vector<double>& t, const std::vector<double>& rho,
                   const std::vector<double>& D, std::vector<double>& S, std::vector<double>& ev);

// The pencil of an element side with no neighbour and not Dirichlet (a natural boundary,
// Sec. 4.2's "suitable boundary conditions"): only the present elements are assembled,
// and the row beyond a free side is decoupled (K = M = 1). S[row*P + mode], S^T M S = I.
void pencil_variant_tables(int n, const std::vector<double>& rho, const std::vector<double>& D, bool low_free,
                           bool high_free, std::vector<double>& S, std::vector<double>& ev);
// Per element: bit 2a (low side) and bit 2a+1 (high side) set when that side along axis a
// has no neighbour and its face is not wholly masked.
std::vector<uint8_t> free_sides(const Numbering& nb, const std::vector<uint8_t>& mask);

// Mean length of the 4 element edges along xi, eta, zeta: hbox[e*3 + axis].
std::vector<double> box_sizes(const Numbering& nb, const double* xyz);

// Physical coordinates of each DOF: xyz of the trilinear map at its owner node.
std::vector<double> dof_coords(const Numbering& nb, const double* xyz, const std::vector<double>& t,
                               const std::vector<int>& owner);

// Q1 coarse matrix (the operator at n = 1, 2-point GLL) on all input vertices.
Csr coarse_matrix(const Numbering& nb, const double* xyz, double lambda);

// Symmetric Jacobi eigen-solver for a dense n x n matrix (row major); eigenvectors in columns.
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& evals, std::vector<double>& evecs);

// Smoothed-aggregation hierarchy (see amg.cpp for the rule).
struct AmgLevel {
  Csr A, P, R;                        // R = P^T
  std::vector<double> dinv;
  // The V(1,1) cycle of this level as two sparse products (smoothed kind only), with
  // Jacobi weight w = kAmgOmega: the pre-smoothing from zero, the residual and the
  // restriction give b_c = M b, M = R (I - w A D^-1); the prolongation and the
  // post-smoothing give x = N b + Q x_c, N = 2w D^-1 - w^2 D^-1 A D^-1, Q = (I - w D^-1 A) P.
  Csr M, N, Q;
};
constexpr double kAmgOmega = 2.0 / 3.0;
struct Amg {
  std::vector<AmgLevel> levels;
  int coarsest_n = 0;
  std::vector<double> coarsest_inv;   // dense, row major
};
// kAmgVcycle: smoothed aggregation (three pairwise passes), applied as three V(1,1) cycles;
// kAmgKcycle: unsmoothed aggregation (two passes, P = T), applied as one K-cycle (Sec. 4.1).
enum AmgKind { kAmgVcycle = 0, kAmgKcycle = 1 };
// Returns "" or an error message (not SPD, stalled).
std::string build_amg(const Csr& A0, Amg& out, int kind = kAmgVcycle);
Csr submatrix(const Csr& A, const std::vector<int>& keep);   // rows/cols in keep, renumbered

}  // namespace sem
