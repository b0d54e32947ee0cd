// Host set-up: GLL tables (Sec. 2.1, 2.4), numbering and gather tables (Sec. 2.2),
// geometry helpers (Sec. 2.3), patch tables and pencil eigen-tables (Sec. 4.2),
// coarse Q1 matrix (Sec. 4.1.1).
#include "host_setup.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

namespace sem {

const int kCornerBits[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                               {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

int corner_of_bits(int a, int b, int c) {
  static const int lut[8] = {0, 1, 3, 2, 4, 5, 7, 6};  // index a + 2b + 4c
  return lut[a + 2 * b + 4 * c];
}

// ---------------------------------------------------------------- GLL tables
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x, d1 = 1.0;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = x * d1 + k * p1;  // P_k' = x P_{k-1}' + k P_{k-1}
    p0 = p1; p1 = p2; d1 = d2;
  }
  p = p1; dp = d1;
}

void gll(int n, std::vector<double>& t, std::vector<double>& rho) {
  t.assign(n + 1, 0.0);
  rho.assign(n + 1, 0.0);
  t[0] = -1.0; t[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    // Newton on P_n'(x) = 0; P_n'' from Legendre's equation.
    double x = -std::cos(M_PI * i / n);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, x, p, dp);
      double ddp = (2.0 * x * dp - n * (n + 1.0) * p) / (1.0 - x * x);
      double dx = dp / ddp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    t[i] = x;
  }
  for (int i = 0; i <= n; ++i) {
    double p, dp;
    legendre(n, t[i], p, dp);
    rho[i] = 2.0 / (n * (n + 1.0) * p * p);
  }
}

std::vector<double> derivative_matrix(int n, const std::vector<double>& t) {
  int p = n + 1;
  std::vector<double> D(p * p, 0.0), Pn(p);
  for (int i = 0; i < p; ++i) { double d; legendre(n, t[i], Pn[i], d); }
  for (int i = 0; i < p; ++i)
    for (int m = 0; m < p; ++m)
      if (i != m) D[i * p + m] = Pn[i] / (Pn[m] * (t[i] - t[m]));
  D[0] = -n * (n + 1.0) / 4.0;
  D[n * p + n] = n * (n + 1.0) / 4.0;
  return D;
}

// ------------------------------------------------------------------ numbering
namespace {

struct FaceKey {
  std::array<int, 4> v;
  bool operator==(const FaceKey& o) const { return v == o.v; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int x : k.v) { h ^= (uint64_t)(uint32_t)x; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  auto spread = [](uint64_t a) {
    a &= 0x1fffff;
    a = (a | a << 32) & 0x1f00000000ffffull;
    a = (a | a << 16) & 0x1f0000ff0000ffull;
    a = (a | a << 8) & 0x100f00f00f00f00full;
    a = (a | a << 4) & 0x10c30c30c30c30c3ull;
    a = (a | a << 2) & 0x1249249249249249ull;
    return a;
  };
  return spread(x) | spread(y) << 1 | spread(z) << 2;
}

// free axes of a face with normal axis d, in increasing order
inline void face_axes(int d, int& u, int& v) {
  u = (d == 0) ? 1 : 0;
  v = (d == 2) ? 1 : 2;
}

struct FaceFrame {
  int cu, cv;      // bits (along u, v) of the corner with the smallest vertex id
  bool first_u;    // canonical first axis is u
};

// Canonical frame of a face from the vertex ids of its corners vid[cu][cv]:
// origin at the smallest id, first axis toward the smaller of its two neighbours.
inline FaceFrame face_frame(const int vid[2][2]) {
  FaceFrame f{0, 0, true};
  int best = vid[0][0];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      if (vid[a][b] < best) { best = vid[a][b]; f.cu = a; f.cv = b; }
  f.first_u = vid[1 - f.cu][f.cv] < vid[f.cu][1 - f.cv];
  return f;
}

inline void face_vids(const int* hv, int d, int s, int out[2][2]) {
  int u, v;
  face_axes(d, u, v);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int bits[3];
      bits[d] = s; bits[u] = a; bits[v] = b;
      out[a][b] = hv[corner_of_bits(bits[0], bits[1], bits[2])];
    }
}

inline void to_canonical(const FaceFrame& f, int n, int a, int b, int& s, int& t) {
  int du = f.cu ? n - a : a, dv = f.cv ? n - b : b;
  if (f.first_u) { s = du; t = dv; } else { s = dv; t = du; }
}
inline void from_canonical(const FaceFrame& f, int n, int s, int t, int& a, int& b) {
  int du = f.first_u ? s : t, dv = f.first_u ? t : s;
  a = f.cu ? n - du : du;
  b = f.cv ? n - dv : dv;
}

}  // namespace

std::string number_mesh(const double* xyz, int64_t nv, const int64_t* hex, int64_t ne, int n,
                        Numbering& out) {
  const int p = n + 1, p3 = p * p * p;
  out.n = n; out.p = p; out.ne = ne; out.nv = nv;
  for (int64_t i = 0; i < 8 * ne; ++i)
    if (hex[i] < 0 || hex[i] >= nv) return "hex2vert entry out of range";
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 8; ++a)
      for (int b = a + 1; b < 8; ++b)
        if (hex[8 * e + a] == hex[8 * e + b]) return "hex with a repeated vertex";

  // library element order: Morton order of centroids (locality of the gathers)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nv; ++v)
    for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], xyz[3 * v + c]); hi[c] = std::max(hi[c], xyz[3 * v + c]); }
  std::vector<uint64_t> code(ne);
  for (int64_t e = 0; e < ne; ++e) {
    double cen[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < 3; ++k) cen[k] += xyz[3 * hex[8 * e + c] + k] / 8.0;
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double s = (hi[k] > lo[k]) ? (cen[k] - lo[k]) / (hi[k] - lo[k]) : 0.0;
      q[k] = (uint32_t)std::min(2097151.0, std::max(0.0, s * 2097151.0));
    }
    code[e] = morton3(q[0], q[1], q[2]);
  }
  out.elem_perm.resize(ne);
  std::iota(out.elem_perm.begin(), out.elem_perm.end(), 0);
  std::stable_sort(out.elem_perm.begin(), out.elem_perm.end(),
                   [&](int64_t a, int64_t b) { return code[a] < code[b]; });
  out.hexv.resize(8 * ne);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 8; ++c) out.hexv[8 * e + c] = (int)hex[8 * out.elem_perm[e] + c];

  // entities: edges keyed by (min, max) vertex ids, faces by sorted corner ids
  std::unordered_map<uint64_t, int> edge_id;
  edge_id.reserve(4 * ne);
  std::unordered_map<FaceKey, int, FaceKeyHash> face_id;
  face_id.reserve(4 * ne);
  std::vector<int> elem_face(6 * ne), elem_edge(12 * ne);
  std::vector<std::vector<std::pair<int, int>>> face_inc;   // (element, face index)
  for (int64_t e = 0; e < ne; ++e) {
    const int* hv = &out.hexv[8 * e];
    int ei = 0;
    for (int a = 0; a < 3; ++a)
      for (int b1 = 0; b1 < 2; ++b1)
        for (int b2 = 0; b2 < 2; ++b2) {
          int bits0[3], bits1[3];
          int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
          bits0[a] = 0; bits1[a] = 1;
          bits0[o1] = bits1[o1] = b1;
          bits0[o2] = bits1[o2] = b2;
          int vA = hv[corner_of_bits(bits0[0], bits0[1], bits0[2])];
          int vB = hv[corner_of_bits(bits1[0], bits1[1], bits1[2])];
          uint64_t key = ((uint64_t)std::min(vA, vB) << 32) | (uint32_t)std::max(vA, vB);
          auto it = edge_id.emplace(key, (int)edge_id.size()).first;
          elem_edge[12 * e + ei++] = it->second;
        }
    for (int f = 0; f < 6; ++f) {
      int vid[2][2];
      face_vids(hv, f / 2, f % 2, vid);
      FaceKey k{{vid[0][0], vid[0][1], vid[1][0], vid[1][1]}};
      std::sort(k.v.begin(), k.v.end());
      auto it = face_id.emplace(k, (int)face_id.size());
      if (it.second) face_inc.emplace_back();
      int fid = it.first->second;
      elem_face[6 * e + f] = fid;
      face_inc[fid].emplace_back((int)e, f);
      if (face_inc[fid].size() > 2) return "non-manifold mesh: a face is shared by more than two hexes";
    }
  }
  const int64_t nedge = (int64_t)edge_id.size(), nface = (int64_t)face_id.size();
  const int64_t m1 = n - 1;
  const int64_t off_edge = nv, off_face = nv + nedge * m1, off_int = off_face + nface * m1 * m1;
  const int64_t Gprov = off_int + ne * m1 * m1 * m1;
  if (Gprov >= (int64_t)1 << 31 || ne * p3 >= (int64_t)1 << 31) return "mesh too large for 32-bit indices";

  // element-interior nodes first, element by element in local order (DOF e m^3 + a +
  // m (b + m c) for local node (a+1, b+1, c+1)), so that their gathers need no index
  // table; then the shared nodes by provisional id per entity, renumbered by first touch
  // in element order
  const int64_t Gi = ne * m1 * m1 * m1;
  std::vector<int> newid(off_int, -1);
  out.l2g.assign(ne * p3, -1);
  int next = (int)Gi;
  std::vector<int64_t> prov(p3);
  for (int64_t e = 0; e < ne; ++e) {
    const int* hv = &out.hexv[8 * e];
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) {
          int idx[3] = {i, j, k};
          int nin = 0, ia = -1;
          for (int a = 0; a < 3; ++a)
            if (idx[a] > 0 && idx[a] < n) { ++nin; ia = a; }
          int64_t id;
          if (nin == 0) {
            id = hv[corner_of_bits(i / n, j / n, k / n)];
          } else if (nin == 1) {
            int o1 = (ia + 1) % 3, o2 = (ia + 2) % 3;
            int b1 = idx[o1] / n, b2 = idx[o2] / n;
            int eidx = 4 * ia + 2 * b1 + b2;
            int bits0[3], bits1[3];
            bits0[ia] = 0; bits1[ia] = 1;
            bits0[o1] = bits1[o1] = b1;
            bits0[o2] = bits1[o2] = b2;
            int vA = hv[corner_of_bits(bits0[0], bits0[1], bits0[2])];
            int vB = hv[corner_of_bits(bits1[0], bits1[1], bits1[2])];
            int t = idx[ia];
            int tc = (vA < vB) ? t : n - t;
            id = off_edge + (int64_t)elem_edge[12 * e + eidx] * m1 + (tc - 1);
          } else if (nin == 2) {
            int d = 0;
            for (int a = 0; a < 3; ++a)
              if (!(idx[a] > 0 && idx[a] < n)) d = a;
            int s = idx[d] / n, u, v;
            face_axes(d, u, v);
            int vid[2][2];
            face_vids(hv, d, s, vid);
            FaceFrame fr = face_frame(vid);
            int cs, ct;
            to_canonical(fr, n, idx[u], idx[v], cs, ct);
            id = off_face + (int64_t)elem_face[6 * e + 2 * d + s] * m1 * m1 + (cs - 1) * m1 + (ct - 1);
          } else {
            out.l2g[e * p3 + i + p * (j + p * k)] = (int)(e * m1 * m1 * m1 + ((i - 1) + m1 * ((j - 1) + m1 * (k - 1))));
            continue;
          }
          int l = i + p * (j + p * k);
          if (newid[id] < 0) newid[id] = next++;
          out.l2g[e * p3 + l] = newid[id];
        }
  }
  out.G = next;
  out.Gi = Gi;

  // vertex DOFs, face neighbours, boundary nodes
  out.vert_dof.assign(nv, -1);
  for (int64_t e = 0; e < ne; ++e)
    for (int c = 0; c < 8; ++c) {
      int l = kCornerBits[c][0] * n + p * (kCornerBits[c][1] * n + p * kCornerBits[c][2] * n);
      out.vert_dof[out.hexv[8 * e + c]] = out.l2g[e * p3 + l];
    }
  out.face_elem.assign(6 * ne, -1);
  out.face_idx.assign(6 * ne, -1);
  out.boundary.assign(out.G, 0);
  for (auto& inc : face_inc) {
    if (inc.size() == 2) {
      out.face_elem[6 * inc[0].first + inc[0].second] = inc[1].first;
      out.face_idx[6 * inc[0].first + inc[0].second] = inc[1].second;
      out.face_elem[6 * inc[1].first + inc[1].second] = inc[0].first;
      out.face_idx[6 * inc[1].first + inc[1].second] = inc[0].second;
    } else {
      int e = inc[0].first, f = inc[0].second, d = f / 2, s = f % 2, u, v;
      face_axes(d, u, v);
      for (int a = 0; a <= n; ++a)
        for (int b = 0; b <= n; ++b) {
          int idx[3];
          idx[d] = s * n; idx[u] = a; idx[v] = b;
          out.boundary[out.l2g[(int64_t)e * p3 + idx[0] + p * (idx[1] + p * idx[2])]] = 1;
        }
    }
  }
  return "";
}

void gather_csr(const Numbering& nb, std::vector<int>& off, std::vector<int>& idx,
                std::vector<int>& owner) {
  const int64_t L = (int64_t)nb.l2g.size();
  off.assign(nb.G + 1, 0);
  for (int64_t l = 0; l < L; ++l) off[nb.l2g[l] + 1]++;
  for (int64_t g = 0; g < nb.G; ++g) off[g + 1] += off[g];
  idx.assign(L, 0);
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int64_t l = 0; l < L; ++l) idx[fill[nb.l2g[l]]++] = (int)l;
  owner.resize(nb.G);
  for (int64_t g = 0; g < nb.G; ++g) owner[g] = idx[off[g]];
}

namespace {

// Global DOF at the virtual local coordinate c (entries in -1..n+1) of element e: the
// element's own node when all entries are in 0..n; otherwise, for the first axis outside,
// the point carried across that face into the neighbour, one layer inside it, and resolved
// there (each step brings one axis inside, so at most three steps); -1 across a face
// without a neighbour.
int virtual_node(const Numbering& nb, int64_t e, const int c[3]) {
  const int n = nb.n, p = nb.p;
  for (int d1 = 0; d1 < 3; ++d1) {
    if (c[d1] >= 0 && c[d1] <= n) continue;
    const int s1 = c[d1] > n ? 1 : 0, f = 2 * d1 + s1;
    const int e2 = nb.face_elem[6 * e + f];
    if (e2 < 0) return -1;
    const int f2 = nb.face_idx[6 * e + f];
    int u1, v1, d2 = f2 / 2, s2 = f2 % 2, u2, v2;
    face_axes(d1, u1, v1);
    face_axes(d2, u2, v2);
    int vid1[2][2], vid2[2][2];
    face_vids(&nb.hexv[8 * e], d1, s1, vid1);
    face_vids(&nb.hexv[8 * (int64_t)e2], d2, s2, vid2);
    int cs, ct, a2, b2;
    to_canonical(face_frame(vid1), n, c[u1], c[v1], cs, ct);   // affine, so valid outside 0..n too
    from_canonical(face_frame(vid2), n, cs, ct, a2, b2);
    int c2[3];
    c2[d2] = s2 ? n - 1 : 1;
    c2[u2] = a2;
    c2[v2] = b2;
    return virtual_node(nb, e2, c2);
  }
  return nb.l2g[e * p * p * p + c[0] + p * (c[1] + p * c[2])];
}

}  // namespace

std::vector<int> patch_table(const Numbering& nb, bool full) {
  const int n = nb.n, p = nb.p, P = n + 3, P3 = P * P * P, p3 = p * p * p;
  const int64_t ne = nb.ne;
  std::vector<int> ip((size_t)ne * P3, -1);
  auto ext = [&](int I, int J, int K) { return (I + 1) + P * ((J + 1) + P * (K + 1)); };
  for (int64_t e = 0; e < ne; ++e) {
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i)
          ip[e * P3 + ext(i, j, k)] = nb.l2g[e * p3 + i + p * (j + p * k)];
    for (int f = 0; f < 6; ++f) {
      int e2 = nb.face_elem[6 * e + f];
      if (e2 < 0) continue;
      int f2 = nb.face_idx[6 * e + f];
      int d1 = f / 2, s1 = f % 2, u1, v1, d2 = f2 / 2, s2 = f2 % 2, u2, v2;
      face_axes(d1, u1, v1);
      face_axes(d2, u2, v2);
      int vid1[2][2], vid2[2][2];
      face_vids(&nb.hexv[8 * e], d1, s1, vid1);
      face_vids(&nb.hexv[8 * e2], d2, s2, vid2);
      FaceFrame fr1 = face_frame(vid1), fr2 = face_frame(vid2);
      for (int a1 = 0; a1 <= n; ++a1)
        for (int b1 = 0; b1 <= n; ++b1) {
          int cs, ct, a2, b2;
          to_canonical(fr1, n, a1, b1, cs, ct);
          from_canonical(fr2, n, cs, ct, a2, b2);
          int c2[3];
          c2[d2] = s2 ? n - 1 : 1; c2[u2] = a2; c2[v2] = b2;
          int g = nb.l2g[(int64_t)e2 * p3 + c2[0] + p * (c2[1] + p * c2[2])];
          int c1[3];
          c1[d1] = s1 ? n + 1 : -1; c1[u1] = a1; c1[v1] = b1;
          ip[e * P3 + ext(c1[0], c1[1], c1[2])] = g;
        }
    }
    if (!full) continue;
    for (int K = -1; K <= n + 1; ++K)
      for (int J = -1; J <= n + 1; ++J)
        for (int I = -1; I <= n + 1; ++I) {
          const int outside = (I < 0 || I > n) + (J < 0 || J > n) + (K < 0 || K > n);
          if (outside < 2) continue;
          const int c[3] = {I, J, K};
          ip[e * P3 + ext(I, J, K)] = virtual_node(nb, e, c);
        }
  }
  return ip;
}

// ------------------------------------------------------------ pencil tables
void pencil_variant_tables(int n, const std::vector<double>& rho, const std::vector<double>& D, bool low_free,
                           bool high_free, std::vector<double>& S, std::vector<double>& ev) {
  const int p = n + 1, P = n + 3;
  std::vector<double> d(p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int m = 0; m < p; ++m) d[i * p + j] += rho[m] * D[m * p + i] * D[m * p + j];
  // box rows 0..P-1 are pencil rows -1..n+1
  std::vector<double> K(P * P, 0.0), M(P, 0.0);
  for (int i = 0; i < p; ++i) {
    M[i + 1] += rho[i];
    for (int j = 0; j < p; ++j) K[(i + 1) * P + (j + 1)] += d[i * p + j];
  }
  if (low_free) {
    K[0] = 1.0;
    M[0] = 1.0;
  } else {   // left neighbour: its nodes n-1, n on rows -1, 0
    K[0] += d[(n - 1) * p + (n - 1)];
    K[0 * P + 1] += d[(n - 1) * p + n];
    K[1 * P + 0] += d[n * p + (n - 1)];
    K[1 * P + 1] += d[n * p + n];
    M[0] += rho[n - 1];
    M[1] += rho[n];
  }
  if (high_free) {
    K[(P - 1) * P + (P - 1)] = 1.0;
    M[P - 1] = 1.0;
  } else {   // right neighbour: its nodes 0, 1 on rows n, n+1
    K[(P - 2) * P + (P - 2)] += d[0];
    K[(P - 2) * P + (P - 1)] += d[1];
    K[(P - 1) * P + (P - 2)] += d[p];
    K[(P - 1) * P + (P - 1)] += d[p + 1];
    M[P - 2] += rho[0];
    M[P - 1] += rho[1];
  }
  // K S = M S diag(ev): eigenpairs of M^-1/2 K M^-1/2, S = M^-1/2 Q
  std::vector<double> A(P * P), Q, vals;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) A[i * P + j] = K[i * P + j] / std::sqrt(M[i] * M[j]);
  jacobi_eigen(P, A, vals, Q);
  S.assign(P * P, 0.0);
  ev = vals;
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c) S[r * P + c] = Q[r * P + c] / std::sqrt(M[r]);
}

std::vector<uint8_t> free_sides(const Numbering& nb, const std::vector<uint8_t>& mask) {
  const int n = nb.n, p = nb.p, p3 = p * p * p;
  std::vector<uint8_t> out(nb.ne, 0);
  for (int64_t e = 0; e < nb.ne; ++e)
    for (int f = 0; f < 6; ++f) {
      if (nb.face_elem[6 * e + f] >= 0) continue;
      const int a = f / 2, side = f % 2;
      bool all_masked = true;
      for (int u = 0; u < p && all_masked; ++u)
        for (int v = 0; v < p && all_masked; ++v) {
          int c[3];
          c[a] = side ? n : 0;
          c[(a + 1) % 3] = u;
          c[(a + 2) % 3] = v;
          if (!mask[nb.l2g[e * p3 + c[0] + p * (c[1] + p * c[2])]]) all_masked = false;
        }
      if (!all_masked) out[e] |= (uint8_t)(1u << (2 * a + side));
    }
  return out;
}
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& evals, std::vector<double>& evecs) {
  evecs.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) evecs[i * n + i] = 1.0;
  double scale = 0.0;
  for (double a : A) scale = std::max(scale, std::fabs(a));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (std::sqrt(off) <= 1e-15 * scale * 1e-3) break;
    for (int pi = 0; pi < n; ++pi)
      for (int q = pi + 1; q < n; ++q) {
        double apq = A[pi * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[pi * n + pi], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // A <- J^T A J, rotation in the (pi, q) plane
          double akp = A[k * n + pi], akq = A[k * n + q];
          A[k * n + pi] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[pi * n + k], aqk = A[q * n + k];
          A[pi * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = evecs[k * n + pi], vkq = evecs[k * n + q];
          evecs[k * n + pi] = c * vkp - s * vkq;
          evecs[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  evals.resize(n);
  for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
}

void pencil_tables(int n, const std::vector<double>& t, const std::vector<double>& rho,
                   const std::vector<double>& D, std::vector<double>& S, std::vector<double>& ev) {
  (void)t;
  const int p = n + 1, P = n + 3;
  std::vector<double> d(p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int m = 0; m < p; ++m) d[i * p + j] += rho[m] * D[m * p + i] * D[m * p + j];
  // rows/cols -1..n+1 of the three-element assembly (Dirichlet beyond them)
  std::vector<double> K(P * P, 0.0), M(P, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) K[(i + 1) * P + (j + 1)] = d[i * p + j];
  K[1 * P + 1] += d[n * p + n];                 // left neighbour's node n sits on 0
  K[(n + 1) * P + (n + 1)] += d[0];             // right neighbour's node 0 sits on n
  K[0] = d[(n - 1) * p + (n - 1)];
  K[0 * P + 1] = K[1 * P + 0] = d[(n - 1) * p + n];
  K[(P - 1) * P + (P - 1)] = d[1 * p + 1];
  K[(P - 1) * P + (P - 2)] = K[(P - 2) * P + (P - 1)] = d[1 * p + 0];
  for (int i = 0; i < p; ++i) M[i + 1] = rho[i];
  M[1] += rho[n];
  M[n + 1] += rho[0];
  M[0] = rho[n - 1];
  M[P - 1] = rho[1];
  // K and M are symmetric under the reflection i -> P-1-i, so the eigenvectors split
  // into even and odd ones. Solve the two half-size problems on the bases
  // e_i + e_{P-1-i} (and e_mid) and e_i - e_{P-1-i}; modes are stored even first.
  const int H = P / 2, odd = P & 1, NE = H + odd;
  auto half_problem = [&](bool even, int m, std::vector<double>& vals, std::vector<double>& vecs) {
    std::vector<double> Kh(m * m), Mh(m);
    auto basis = [&](int i, int row) -> double {   // entry `row` of basis vector i
      if (even && odd && i == H) return row == H ? 1.0 : 0.0;
      if (row == i) return 1.0;
      if (row == P - 1 - i) return even ? 1.0 : -1.0;
      return 0.0;
    };
    for (int i = 0; i < m; ++i) {
      double mi = 0.0;
      for (int r = 0; r < P; ++r) mi += basis(i, r) * M[r] * basis(i, r);
      Mh[i] = mi;
      for (int j = 0; j < m; ++j) {
        double kij = 0.0;
        for (int r = 0; r < P; ++r)
          for (int c = 0; c < P; ++c) kij += basis(i, r) * K[r * P + c] * basis(j, c);
        Kh[i * m + j] = kij;
      }
    }
    std::vector<double> A(m * m), Q;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[i * m + j] = Kh[i * m + j] / std::sqrt(Mh[i] * Mh[j]);
    jacobi_eigen(m, A, vals, Q);
    vecs.assign(P * m, 0.0);   // full-length eigenvectors, column a
    for (int a = 0; a < m; ++a)
      for (int i = 0; i < m; ++i) {
        const double y = Q[i * m + a] / std::sqrt(Mh[i]);
        for (int r = 0; r < P; ++r) vecs[r * m + a] += basis(i, r) * y;
      }
  };
  std::vector<double> ev_e, S_e, ev_o, S_o;
  half_problem(true, NE, ev_e, S_e);
  half_problem(false, H, ev_o, S_o);
  S.assign(P * P, 0.0);
  ev.assign(P, 0.0);
  for (int a = 0; a < NE; ++a) {
    ev[a] = ev_e[a];
    for (int r = 0; r < P; ++r) S[r * P + a] = S_e[r * NE + a];
  }
  for (int a = 0; a < H; ++a) {
    ev[NE + a] = ev_o[a];
    for (int r = 0; r < P; ++r) S[r * P + NE + a] = S_o[r * H + a];
  }
}

std::vector<double> box_sizes(const Numbering& nb, const double* xyz) {
  std::vector<double> h(3 * nb.ne, 0.0);
  for (int64_t e = 0; e < nb.ne; ++e)
    for (int ax = 0; ax < 3; ++ax) {
      double s = 0.0;
      for (int c = 0; c < 8; ++c) {
        if (kCornerBits[c][ax] != 0) continue;
        int b[3] = {kCornerBits[c][0], kCornerBits[c][1], kCornerBits[c][2]};
        b[ax] = 1;
        int c2 = corner_of_bits(b[0], b[1], b[2]);
        const double* x0 = &xyz[3 * nb.hexv[8 * e + c]];
        const double* x1 = &xyz[3 * nb.hexv[8 * e + c2]];
        s += std::sqrt((x1[0] - x0[0]) * (x1[0] - x0[0]) + (x1[1] - x0[1]) * (x1[1] - x0[1]) +
                       (x1[2] - x0[2]) * (x1[2] - x0[2]));
      }
      h[3 * e + ax] = s / 4.0;
    }
  return h;
}

std::vector<double> dof_coords(const Numbering& nb, const double* xyz, const std::vector<double>& t,
                               const std::vector<int>& owner) {
  const int p = nb.p, p3 = p * p * p;
  std::vector<double> X(3 * nb.G);
  for (int64_t g = 0; g < nb.G; ++g) {
    int l = owner[g];
    int64_t e = l / p3;
    int r = l % p3, i = r % p, j = (r / p) % p, k = r / (p * p);
    double x[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
      double N = (kCornerBits[c][0] ? 1 + t[i] : 1 - t[i]) * (kCornerBits[c][1] ? 1 + t[j] : 1 - t[j]) *
                 (kCornerBits[c][2] ? 1 + t[k] : 1 - t[k]) / 8.0;
      for (int a = 0; a < 3; ++a) x[a] += N * xyz[3 * nb.hexv[8 * e + c] + a];
    }
    for (int a = 0; a < 3; ++a) X[3 * g + a] = x[a];
  }
  return X;
}

// ------------------------------------------------------------ coarse matrix
Csr coarse_matrix(const Numbering& nb, const double* xyz, double lambda) {
  // Operator of Eq. R at n = 1: nodes are the corners (t = -1, +1), weights 1,
  // Dhat[i][m] = phi_m'(t_i) = (-1/2, +1/2) for both i.
  const double Dh[2][2] = {{-0.5, 0.5}, {-0.5, 0.5}};
  std::vector<std::array<double, 3>> trip;  // (row, col, val) packed below
  std::vector<int64_t> rows, cols;
  std::vector<double> vals;
  rows.reserve(64 * nb.ne); cols.reserve(64 * nb.ne); vals.reserve(64 * nb.ne);
  for (int64_t e = 0; e < nb.ne; ++e) {
    double Gf[8][6], m[8];
    for (int q = 0; q < 8; ++q) {   // local node q = i + 2(j + 2k)
      int qi = q & 1, qj = (q >> 1) & 1, qk = q >> 2;
      double tq[3] = {qi ? 1.0 : -1.0, qj ? 1.0 : -1.0, qk ? 1.0 : -1.0};
      double J[3][3] = {{0}};
      for (int c = 0; c < 8; ++c) {
        double s[3] = {kCornerBits[c][0] ? 1.0 : -1.0, kCornerBits[c][1] ? 1.0 : -1.0, kCornerBits[c][2] ? 1.0 : -1.0};
        double f[3] = {(1 + s[0] * tq[0]) / 2, (1 + s[1] * tq[1]) / 2, (1 + s[2] * tq[2]) / 2};
        double dN[3] = {s[0] / 2 * f[1] * f[2], f[0] * s[1] / 2 * f[2], f[0] * f[1] * s[2] / 2};
        const double* xv = &xyz[3 * nb.hexv[8 * e + c]];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) J[a][b] += xv[a] * dN[b];
      }
      double C[3][3];   // cofactor matrix: inv(J) = C^T / det
      C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
      // G = det * inv(J) inv(J)^T = (C^T C) / det ; inv(J)[a][b] = C[b][a] / det
      double Gm[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double s = 0;
          for (int c = 0; c < 3; ++c) s += C[c][a] * C[c][b];
          Gm[a][b] = s / det;
        }
      Gf[q][0] = Gm[0][0]; Gf[q][1] = Gm[0][1]; Gf[q][2] = Gm[0][2];
      Gf[q][3] = Gm[1][1]; Gf[q][4] = Gm[1][2]; Gf[q][5] = Gm[2][2];
      m[q] = det;
    }
    for (int b = 0; b < 8; ++b) {
      double u[8] = {0};
      u[b] = 1.0;
      double A[8], B[8], Cc[8];
      for (int q = 0; q < 8; ++q) {
        int i = q & 1, j = (q >> 1) & 1, k = q >> 2;
        double ur = 0, us = 0, ut = 0;
        for (int mm = 0; mm < 2; ++mm) {
          ur += Dh[i][mm] * u[mm + 2 * (j + 2 * k)];
          us += Dh[j][mm] * u[i + 2 * (mm + 2 * k)];
          ut += Dh[k][mm] * u[i + 2 * (j + 2 * mm)];
        }
        A[q] = Gf[q][0] * ur + Gf[q][1] * us + Gf[q][2] * ut;
        B[q] = Gf[q][1] * ur + Gf[q][3] * us + Gf[q][4] * ut;
        Cc[q] = Gf[q][2] * ur + Gf[q][4] * us + Gf[q][5] * ut;
      }
      for (int q = 0; q < 8; ++q) {
        int i = q & 1, j = (q >> 1) & 1, k = q >> 2;
        double r = 0;
        for (int mm = 0; mm < 2; ++mm) {
          r += Dh[mm][i] * A[mm + 2 * (j + 2 * k)];
          r += Dh[mm][j] * B[i + 2 * (mm + 2 * k)];
          r += Dh[mm][k] * Cc[i + 2 * (j + 2 * mm)];
        }
        r += lambda * m[q] * u[q];
        int va = nb.hexv[8 * e + corner_of_bits(i, j, k)];
        int vb = nb.hexv[8 * e + corner_of_bits(b & 1, (b >> 1) & 1, b >> 2)];
        rows.push_back(va); cols.push_back(vb); vals.push_back(r);
      }
    }
  }
  // sort triplets by (row, col) keeping element order for equal keys, then sum
  std::vector<int64_t> ord(rows.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    return rows[a] != rows[b] ? rows[a] < rows[b] : cols[a] < cols[b];
  });
  Csr A;
  A.n = A.m = (int)nb.nv;
  A.ptr.assign(A.n + 1, 0);
  int64_t prev_r = -1, prev_c = -1;
  for (int64_t o : ord) {
    if (rows[o] == prev_r && cols[o] == prev_c) {
      A.val.back() += vals[o];
    } else {
      A.col.push_back((int)cols[o]);
      A.val.push_back(vals[o]);
      A.ptr[rows[o] + 1]++;
      prev_r = rows[o]; prev_c = cols[o];
    }
  }
  for (int i = 0; i < A.n; ++i) A.ptr[i + 1] += A.ptr[i];
  return A;
}

Csr submatrix(const Csr& A, const std::vector<int>& keep) {
  std::vector<int> map(A.m, -1);
  for (size_t i = 0; i < keep.size(); ++i) map[keep[i]] = (int)i;
  Csr B;
  B.n = B.m = (int)keep.size();
  B.ptr.assign(B.n + 1, 0);
  for (int r = 0; r < B.n; ++r) {
    int i = keep[r];
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (map[A.col[q]] >= 0) { B.col.push_back(map[A.col[q]]); B.val.push_back(A.val[q]); }
    B.ptr[r + 1] = (int)B.col.size();
  }
  return B;   // columns stay sorted: map is increasing on keep (ascending)
}

}  // namespace sem
