// Smoothed-aggregation AMG hierarchy for the coarse solve P_0 (Sec. 4.1.1).
//
// The paper names aggregation AMG with a K-cycle and damped Jacobi without
// defining the aggregation; this library uses a fixed, linear, symmetric rule:
//  * pairwise pass over unknowns in increasing order: an unaggregated i joins the
//    unaggregated neighbour j with the largest s = -a_ij among a_ij < 0 and
//    s >= 0.25 max_k(-a_ik); a later j replaces the choice only when its s is
//    larger by a factor 1 + 1e-10 (near-ties keep the lowest j); otherwise i is a
//    singleton; aggregates are numbered in creation order;
//  * three pairwise passes per level (each on the Galerkin product of the last)
//    give tentative aggregates T of up to 8 unknowns;
//  * P = (I - w_P D^{-1} A) T, w_P = (4/3) / max_i(sum_j |a_ij| / a_ii); A_c = P^T A P;
//  * levels are added while a level has more than 2048 unknowns and the passes
//    shrink it to at most 3/4; the coarsest (at most 4096 unknowns) is inverted
//    densely (Cholesky).
// The cycle applied on the GPU is a symmetric V(1,1) with Jacobi weight 2/3,
// repeated three times as a stationary iteration.
// The paper's own variant (kAmgKcycle): unsmoothed aggregation, i.e. two pairwise passes
// (aggregates of up to 4) and P = T, A_c = T^T A T, applied as one recursive K-cycle.
#include <algorithm>
#include <cmath>
#include <thread>

#include "host_setup.h"

namespace sem {
namespace {

const double kBeta = 0.25, kTie = 1e-10;
const int kMaxCoarsest = 2048, kPasses = 3, kDenseLimit = 4096;
const double kStall = 0.75;

std::vector<int> pairwise(const Csr& A, int& na) {
  std::vector<int> agg(A.n, -1);
  na = 0;
  for (int i = 0; i < A.n; ++i) {
    if (agg[i] >= 0) continue;
    double smax = 0.0;
    bool any = false;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (A.col[q] != i && A.val[q] < 0) { smax = any ? std::max(smax, -A.val[q]) : -A.val[q]; any = true; }
    int best = -1;
    double bv = 0.0;
    if (any) {
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
        int j = A.col[q];
        double v = A.val[q];
        if (j == i || v >= 0 || agg[j] >= 0) continue;
        double s = -v;
        if (s < kBeta * smax) continue;
        if (best < 0 || s > bv * (1.0 + kTie)) { best = j; bv = s; }
      }
    }
    agg[i] = na;
    if (best >= 0) agg[best] = na;
    ++na;
  }
  return agg;
}

// C = A * B (sparse), columns sorted, duplicate columns summed in the order met.
Csr spgemm(const Csr& A, const Csr& B) {
  Csr C;
  C.n = A.n; C.m = B.m;
  C.ptr.assign(C.n + 1, 0);
  std::vector<int> mark(B.m, -1);
  std::vector<int> cols;
  std::vector<double> acc(B.m, 0.0);
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    for (int qa = A.ptr[i]; qa < A.ptr[i + 1]; ++qa) {
      int k = A.col[qa];
      double a = A.val[qa];
      for (int qb = B.ptr[k]; qb < B.ptr[k + 1]; ++qb) {
        int j = B.col[qb];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols.push_back(j); }
        acc[j] += a * B.val[qb];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) { C.col.push_back(j); C.val.push_back(acc[j]); }
    C.ptr[i + 1] = (int)C.col.size();
  }
  return C;
}

Csr transpose(const Csr& A) {
  Csr T;
  T.n = A.m; T.m = A.n;
  T.ptr.assign(T.n + 1, 0);
  for (int c : A.col) T.ptr[c + 1]++;
  for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.n; ++i)   // rows in order -> columns of T sorted
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      int d = fill[A.col[q]]++;
      T.col[d] = i;
      T.val[d] = A.val[q];
    }
  return T;
}

Csr aggregation_matrix(const std::vector<int>& agg, int na) {
  Csr T;
  T.n = (int)agg.size(); T.m = na;
  T.ptr.resize(T.n + 1);
  for (int i = 0; i <= T.n; ++i) T.ptr[i] = i;
  T.col = agg;
  T.val.assign(T.n, 1.0);
  return T;
}

// A with every entry a_ij replaced by f(i, j, a_ij) (same pattern).
template <class F>
Csr map_entries(const Csr& A, F f) {
  Csr B = A;
  for (int i = 0; i < A.n; ++i)
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) B.val[q] = f(i, A.col[q], A.val[q]);
  return B;
}

// M, N, Q of a smoothed level (see AmgLevel). Every row of A holds its diagonal.
void fused_cycle_matrices(AmgLevel& lv) {
  const double w = kAmgOmega;
  const std::vector<double>& di = lv.dinv;
  // I - w A D^-1 and I - w D^-1 A
  Csr Bm = map_entries(lv.A, [&](int i, int j, double a) { return (i == j ? 1.0 : 0.0) - w * a * di[j]; });
  Csr Cm = map_entries(lv.A, [&](int i, int j, double a) { return (i == j ? 1.0 : 0.0) - w * di[i] * a; });
  lv.M = spgemm(lv.R, Bm);
  lv.N = map_entries(lv.A, [&](int i, int j, double a) {
    return (i == j ? 2.0 * w * di[i] : 0.0) - w * w * di[i] * a * di[j];
  });
  lv.Q = spgemm(Cm, lv.P);
}

// Runs f(i) for i in [0, n) on the host cores; each i is done by exactly one thread.
template <class F>
void parallel_for(int n, F f) {
  int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 64) nt = 1;
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([=, &f] {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

}  // namespace

std::string build_amg(const Csr& A0, Amg& out, int kind) {
  out.levels.clear();
  const bool smoothed = (kind == kAmgVcycle);
  const int passes = smoothed ? kPasses : 2;
  Csr A = A0;
  while (A.n > kMaxCoarsest) {
    std::vector<int> agg(A.n);
    for (int i = 0; i < A.n; ++i) agg[i] = i;
    Csr Ac = A;
    int nc = A.n;
    for (int pass = 0; pass < passes; ++pass) {
      int na;
      std::vector<int> a = pairwise(Ac, na);
      for (int i = 0; i < A.n; ++i) agg[i] = a[agg[i]];
      Csr T1 = aggregation_matrix(a, na);
      Ac = spgemm(transpose(T1), spgemm(Ac, T1));
      nc = na;
    }
    if (nc > kStall * A.n) break;
    Csr T = aggregation_matrix(agg, nc);
    std::vector<double> d(A.n, 0.0);
    double gersh = 0.0;
    for (int i = 0; i < A.n; ++i) {
      double rs = 0.0;
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
        if (A.col[q] == i) d[i] = A.val[q];
        rs += std::fabs(A.val[q]);
      }
      if (!(d[i] > 0)) return "coarse matrix has a non-positive diagonal";
      gersh = std::max(gersh, rs / d[i]);
    }
    AmgLevel lv;
    if (!smoothed) {
      lv.A = A;
      lv.P = T;
      lv.R = transpose(T);
      lv.dinv.resize(A.n);
      for (int i = 0; i < A.n; ++i) lv.dinv[i] = 1.0 / d[i];
      Csr Anext = spgemm(lv.R, spgemm(A, T));
      out.levels.push_back(std::move(lv));
      A = std::move(Anext);
      continue;
    }
    const double wP = (4.0 / 3.0) / gersh;
    Csr AT = spgemm(A, T);
    // P = T - wP D^{-1} (A T), exact zeros dropped
    Csr P;
    P.n = A.n; P.m = nc;
    P.ptr.assign(P.n + 1, 0);
    for (int i = 0; i < A.n; ++i) {
      bool placed = false;
      for (int q = AT.ptr[i]; q < AT.ptr[i + 1]; ++q) {
        int j = AT.col[q];
        double v = -wP * AT.val[q] / d[i];
        if (j == agg[i]) { v += 1.0; placed = true; }
        if (v != 0.0) { P.col.push_back(j); P.val.push_back(v); }
      }
      if (!placed) {   // T entry whose column is absent from A T (cannot happen for a_ii > 0)
        auto pos = std::lower_bound(P.col.begin() + P.ptr[i], P.col.end(), agg[i]) - P.col.begin();
        P.col.insert(P.col.begin() + pos, agg[i]);
        P.val.insert(P.val.begin() + pos, 1.0);
      }
      P.ptr[i + 1] = (int)P.col.size();
    }
    lv.A = A;
    lv.P = P;
    lv.R = transpose(P);
    lv.dinv.resize(A.n);
    for (int i = 0; i < A.n; ++i) lv.dinv[i] = 1.0 / d[i];
    fused_cycle_matrices(lv);
    Csr Anext = spgemm(lv.R, spgemm(A, P));
    out.levels.push_back(std::move(lv));
    A = std::move(Anext);
  }
  if (A.n > kDenseLimit) return "AMG coarsening stalled above the dense limit";
  // dense Cholesky A = L L^T, inverse = L^{-T} L^{-1}
  const int n = A.n;
  std::vector<double> Ad((size_t)n * n, 0.0), L((size_t)n * n, 0.0), Li((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) Ad[(size_t)i * n + A.col[q]] = A.val[q];
  for (int j = 0; j < n; ++j) {
    double s = Ad[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(s > 0)) return "coarse matrix is not positive definite";
    double ljj = std::sqrt(s);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = Ad[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  // row j of LiT = column j of L^{-1} (forward substitution, contiguous loops)
  std::vector<double>& LiT = Li;
  parallel_for(n, [&](int j) {
    double* y = &LiT[(size_t)j * n];
    for (int i = j; i < n; ++i) {
      const double* Lr = &L[(size_t)i * n];
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= Lr[k] * y[k];
      y[i] = s / Lr[i];
    }
  });
  out.coarsest_n = n;
  out.coarsest_inv.assign((size_t)n * n, 0.0);
  parallel_for(n, [&](int i) {   // inv = L^{-T} L^{-1}: (i, j) = sum_k LiT[i][k] LiT[j][k]
    const double* a = &LiT[(size_t)i * n];
    for (int j = 0; j < n; ++j) {
      const double* b = &LiT[(size_t)j * n];
      double s = 0.0;
      for (int k = std::max(i, j); k < n; ++k) s += a[k] * b[k];
      out.coarsest_inv[(size_t)i * n + j] = s;
    }
  });
  return "";
}

}  // namespace sem
