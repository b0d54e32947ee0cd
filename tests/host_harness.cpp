// Test-only C entry points around the library's host set-up (no CUDA), so the
// numbering, patch tables, pencil tables and AMG hierarchy can be compared with
// the CPU oracle without a GPU. Built by tests/test_host_setup.py.
#include <cstring>
#include <vector>

#include "../paper_1506_05996_gb300/csrc/host_setup.h"

namespace {
sem::Numbering g_nb;
std::vector<int> g_owner, g_off, g_idx, g_ip;
std::vector<double> g_coords, g_hbox, g_S, g_ev, g_t, g_rho, g_D;
sem::Amg g_amg;
std::vector<int> g_keep;
sem::Csr g_A0;
}

extern "C" {

int hh_setup(const double* xyz, int64_t nv, const int64_t* hex, int64_t ne, int n, double lam, int neumann,
             int amg_kind, int patch_full) {
  std::string err = sem::number_mesh(xyz, nv, hex, ne, n, g_nb);
  if (!err.empty()) return -1;
  sem::gll(n, g_t, g_rho);
  g_D = sem::derivative_matrix(n, g_t);
  sem::gather_csr(g_nb, g_off, g_idx, g_owner);
  g_ip = sem::patch_table(g_nb, patch_full != 0);
  sem::pencil_tables(n, g_t, g_rho, g_D, g_S, g_ev);
  g_hbox = sem::box_sizes(g_nb, xyz);
  g_coords = sem::dof_coords(g_nb, xyz, g_t, g_owner);
  sem::Csr A0full = sem::coarse_matrix(g_nb, xyz, lam);
  g_keep.clear();
  for (int64_t v = 0; v < nv; ++v) {
    int g = g_nb.vert_dof[v];
    if (g >= 0 && (neumann || g_nb.boundary[g] == 0)) g_keep.push_back((int)v);
  }
  g_A0 = sem::submatrix(A0full, g_keep);
  err = sem::build_amg(g_A0, g_amg, amg_kind);
  return err.empty() ? 0 : -2;
}

int64_t hh_G() { return g_nb.G; }
void hh_g2l(int* off, int* idx) {
  std::memcpy(off, g_off.data(), g_off.size() * sizeof(int));
  std::memcpy(idx, g_idx.data(), g_idx.size() * sizeof(int));
}
void hh_l2g(int* out) { std::memcpy(out, g_nb.l2g.data(), g_nb.l2g.size() * sizeof(int)); }
void hh_elem_perm(int64_t* out) { std::memcpy(out, g_nb.elem_perm.data(), g_nb.elem_perm.size() * sizeof(int64_t)); }
void hh_coords(double* out) { std::memcpy(out, g_coords.data(), g_coords.size() * sizeof(double)); }
void hh_boundary(uint8_t* out) { std::memcpy(out, g_nb.boundary.data(), g_nb.boundary.size()); }
void hh_ip(int* out) { std::memcpy(out, g_ip.data(), g_ip.size() * sizeof(int)); }
void hh_hbox(double* out) { std::memcpy(out, g_hbox.data(), g_hbox.size() * sizeof(double)); }
void hh_pencil(double* S, double* ev) {
  std::memcpy(S, g_S.data(), g_S.size() * sizeof(double));
  std::memcpy(ev, g_ev.data(), g_ev.size() * sizeof(double));
}
void hh_gll(double* t, double* rho, double* D) {
  std::memcpy(t, g_t.data(), g_t.size() * sizeof(double));
  std::memcpy(rho, g_rho.data(), g_rho.size() * sizeof(double));
  std::memcpy(D, g_D.data(), g_D.size() * sizeof(double));
}
int hh_amg_nlevels() { return (int)g_amg.levels.size(); }
int hh_amg_size(int l) { return l < (int)g_amg.levels.size() ? g_amg.levels[l].A.n : g_amg.coarsest_n; }
static const sem::Csr& amg_mat(int l, int which) {   // which: 0 A, 1 P, 2 M, 3 N, 4 Q
  const sem::AmgLevel& L = g_amg.levels[l];
  switch (which) {
    case 0: return L.A;
    case 1: return L.P;
    case 2: return L.M;
    case 3: return L.N;
    default: return L.Q;
  }
}
int hh_amg_nnz(int l, int which) { return (int)amg_mat(l, which).val.size(); }
int hh_amg_rows(int l, int which) { return amg_mat(l, which).n; }
int hh_amg_cols(int l, int which) { return amg_mat(l, which).m; }
void hh_amg_csr(int l, int which, int* ptr, int* col, double* val) {
  const sem::Csr& A = amg_mat(l, which);
  std::memcpy(ptr, A.ptr.data(), A.ptr.size() * sizeof(int));
  std::memcpy(col, A.col.data(), A.col.size() * sizeof(int));
  std::memcpy(val, A.val.data(), A.val.size() * sizeof(double));
}
void hh_amg_coarsest(double* out) {
  std::memcpy(out, g_amg.coarsest_inv.data(), g_amg.coarsest_inv.size() * sizeof(double));
}
int hh_nkeep() { return (int)g_keep.size(); }
void hh_keep(int* out) { std::memcpy(out, g_keep.data(), g_keep.size() * sizeof(int)); }
}
