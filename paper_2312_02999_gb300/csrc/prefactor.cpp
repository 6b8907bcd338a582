// One-time precomputation of the PD global step (host, C++).
//
// Sec. 2.1 / Eq. 2: H = sum_i w_i G_i^T G_i is constant and is factored once.
// Because each row of F_i depends on one coordinate only, H = K (x) I_3 with
// the scalar matrix K_ab = sum_i w_i gradN_a . gradN_b; every factorisation
// here is done on K (9x less memory, three right-hand sides per solve).
// Sec. 3.1: the free vertices split into x1 (collision-free) and x2
// (collision-aware); H11 = L1 L1^T is the prefactored block and
// Sigma = H22 - H21 H11^-1 H12 (Eq. 9) is dense.  Sec. 3.2 uses Sigma^-1
// explicitly, computed here once.
//
// Layout produced for the GPU: solver positions 0..n1-1 are x1 in a
// nested-dissection order, n1..n1+n2-1 are x2.  Each supernode J of L1 (one
// nested-dissection block) stores Z_J = [L_JJ^-1 ; L_RJ L_JJ^-1] column-major,
// so that a forward solve is y_J = Z_J[:ns] b_J, b_R -= Z_J[ns:] b_J and a
// backward solve is x_J = Z_J^T [y_J ; -x_R].
#include "fsim_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

namespace fsim {

namespace {

constexpr int kLeafSize = 64;

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::max(1u, std::min(hw, 16u));
  if (n < 64 || nt == 1) { body(0, n); return; }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(body, b, e);
  }
  for (auto& x : th) x.join();
}

inline double dot(const double* a, const double* b, int n) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    s0 += a[k] * b[k]; s1 += a[k + 1] * b[k + 1];
    s2 += a[k + 2] * b[k + 2]; s3 += a[k + 3] * b[k + 3];
  }
  for (; k < n; ++k) s0 += a[k] * b[k];
  return (s0 + s1) + (s2 + s3);
}

// Lower Cholesky in place (row-major, leading dimension ld), rows/cols [0,n).
bool potrf_lower(double* A, int n, int64_t ld) {
  for (int j = 0; j < n; ++j) {
    double* aj = A + j * ld;
    double d = aj[j] - dot(aj, aj, j);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    aj[j] = d;
    const double inv = 1.0 / d;
    for (int i = j + 1; i < n; ++i) {
      double* ai = A + i * ld;
      ai[j] = (ai[j] - dot(ai, aj, j)) * inv;
    }
  }
  return true;
}

// Rows [r0,r1) of A (columns [0,ns)) := A L^-T, L lower ns x ns (ld lda).
void trsm_rows(double* A, int64_t ld, int r0, int r1, const double* L, int64_t lda, int ns) {
  for (int i = r0; i < r1; ++i) {
    double* ai = A + (int64_t)i * ld;
    for (int j = 0; j < ns; ++j) {
      const double* lj = L + j * lda;
      ai[j] = (ai[j] - dot(ai, lj, j)) / lj[j];
    }
  }
}

// Inverse of a lower triangular L (n x n, row-major ld) into Li (n x n, row-major).
void trtri_lower(const double* L, int64_t ld, int n, double* Li) {
  std::fill(Li, Li + (int64_t)n * n, 0.0);
  // column j of Li solves L y = e_j; rows i >= j
  for (int j = 0; j < n; ++j) {
    Li[(int64_t)j * n + j] = 1.0 / L[j * ld + j];
    for (int i = j + 1; i < n; ++i) {
      const double* li = L + i * ld;
      double s = 0.0;
      for (int k = j; k < i; ++k) s += li[k] * Li[(int64_t)k * n + j];
      Li[(int64_t)i * n + j] = -s / li[i];
    }
  }
}

struct Graph {
  std::vector<int> ptr, adj;  // symmetric adjacency (no self loops)
};

// --------------------------------------------------------------------------
// geometric nested dissection of the x1 vertices
// --------------------------------------------------------------------------
struct NDBuilder {
  const Graph& g;            // graph on local ids 0..m-1
  const double* xyz;         // coordinates of local ids (3*m)
  std::vector<int> order;    // local ids in elimination order
  std::vector<int> blk_begin, blk_end, blk_parent;
  std::vector<int> stamp, side;
  int call = 0;

  NDBuilder(const Graph& g_, const double* xyz_, int m) : g(g_), xyz(xyz_) {
    stamp.assign(m, -1);
    side.assign(m, 0);
    order.reserve(m);
  }

  int new_block(int b, int e) {
    blk_begin.push_back(b); blk_end.push_back(e); blk_parent.push_back(-1);
    return (int)blk_begin.size() - 1;
  }

  // Orders `v` (appending to order) and returns the root blocks of the subtree.
  std::vector<int> run(std::vector<int> v) {
    if (v.empty()) return {};
    if ((int)v.size() <= kLeafSize) {
      std::sort(v.begin(), v.end());
      int b = (int)order.size();
      for (int u : v) order.push_back(u);
      return {new_block(b, (int)order.size())};
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int u : v)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * u + d]);
        hi[d] = std::max(hi[d], xyz[3 * u + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    // split by rank along the axis (ties broken by id: deterministic)
    std::vector<int> s = v;
    size_t half = s.size() / 2;
    std::nth_element(s.begin(), s.begin() + half, s.end(), [&](int a, int b) {
      double ca = xyz[3 * a + ax], cb = xyz[3 * b + ax];
      return ca < cb || (ca == cb && a < b);
    });
    const int id = call++;
    for (size_t k = 0; k < s.size(); ++k) {
      stamp[s[k]] = id;
      side[s[k]] = k < half ? 0 : 1;
    }
    std::vector<int> left, right, sep;
    for (size_t k = 0; k < s.size(); ++k) {
      int u = s[k];
      if (side[u] == 1) { right.push_back(u); continue; }
      bool cut = false;
      for (int e = g.ptr[u]; e < g.ptr[u + 1]; ++e) {
        int w = g.adj[e];
        if (stamp[w] == id && side[w] == 1) { cut = true; break; }
      }
      (cut ? sep : left).push_back(u);
    }
    std::vector<int> rl = run(std::move(left));
    std::vector<int> rr = run(std::move(right));
    std::vector<int> roots;
    if (sep.empty()) {
      roots = rl;
      roots.insert(roots.end(), rr.begin(), rr.end());
      return roots;
    }
    std::sort(sep.begin(), sep.end());
    int b = (int)order.size();
    for (int u : sep) order.push_back(u);
    int blk = new_block(b, (int)order.size());
    for (int c : rl) blk_parent[c] = blk;
    for (int c : rr) blk_parent[c] = blk;
    return {blk};
  }
};

}  // namespace

void tet_rest_data(const double* rest, const int32_t* tets, int64_t T, double weight_scale,
                   std::vector<double>& dminv, std::vector<double>& w) {
  dminv.assign(9 * T, 0.0);
  w.assign(T, 0.0);
  for (int64_t t = 0; t < T; ++t) {
    const double* X0 = rest + 3 * (int64_t)tets[4 * t + 0];
    double Dm[3][3];
    for (int a = 0; a < 3; ++a) {
      const double* Xa = rest + 3 * (int64_t)tets[4 * t + a + 1];
      for (int d = 0; d < 3; ++d) Dm[d][a] = Xa[d] - X0[d];  // columns X_a - X_0
    }
    double c00 = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
    double c01 = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
    double c02 = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
    double det = Dm[0][0] * c00 + Dm[0][1] * c01 + Dm[0][2] * c02;
    double inv[3][3];
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
    inv[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
    inv[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
    inv[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
    inv[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
    inv[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) dminv[(3 * r + c) * T + t] = inv[r][c];
    w[t] = weight_scale * std::fabs(det) / 6.0;
  }
}

int build_factor(int64_t n, const double* rest, const int32_t* tets, int64_t T,
                 const std::vector<double>& dminv, const std::vector<double>& w,
                 const uint8_t* pinned, const std::vector<uint8_t>& x2mask,
                 HostFactor& f) {
  // ---- free vertices, x1 / x2 split --------------------------------------
  std::vector<int> x1v, x2v;
  for (int64_t v = 0; v < n; ++v) {
    if (pinned[v]) continue;
    (x2mask[v] ? x2v : x1v).push_back((int)v);
  }
  const int n1 = (int)x1v.size(), n2 = (int)x2v.size(), nf = n1 + n2;
  if (nf == 0) return FSIM_EINVAL;
  f.n_free = nf; f.n1 = n1; f.n2 = n2;

  // ---- scalar K over all vertices (triplets -> per-row merge) -------------
  std::vector<std::vector<std::pair<int, double>>> rowsK(n);
  for (int64_t t = 0; t < T; ++t) {
    double gN[4][3];
    for (int a = 1; a < 4; ++a)
      for (int d = 0; d < 3; ++d) gN[a][d] = dminv[(3 * (a - 1) + d) * T + t];
    for (int d = 0; d < 3; ++d) gN[0][d] = -(gN[1][d] + gN[2][d] + gN[3][d]);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double v = w[t] * (gN[a][0] * gN[b][0] + gN[a][1] * gN[b][1] + gN[a][2] * gN[b][2]);
        rowsK[tets[4 * t + a]].push_back({tets[4 * t + b], v});
      }
  }
  for (auto& r : rowsK) {
    std::sort(r.begin(), r.end(), [](auto& a, auto& b) { return a.first < b.first; });
    size_t o = 0;
    for (size_t k = 0; k < r.size(); ++k) {
      if (o > 0 && r[o - 1].first == r[k].first) r[o - 1].second += r[k].second;
      else r[o++] = r[k];
    }
    r.resize(o);
  }

  // ---- nested dissection of x1 ---------------------------------------------
  std::vector<int> loc1(n, -1);
  for (int k = 0; k < n1; ++k) loc1[x1v[k]] = k;
  Graph g1;
  g1.ptr.assign(n1 + 1, 0);
  for (int k = 0; k < n1; ++k) {
    for (auto& e : rowsK[x1v[k]])
      if (e.first != x1v[k] && loc1[e.first] >= 0) g1.adj.push_back(loc1[e.first]);
    g1.ptr[k + 1] = (int)g1.adj.size();
  }
  std::vector<double> xyz1(3 * (size_t)n1);
  for (int k = 0; k < n1; ++k)
    for (int d = 0; d < 3; ++d) xyz1[3 * k + d] = rest[3 * (int64_t)x1v[k] + d];
  NDBuilder nd(g1, xyz1.data(), n1);
  std::vector<int> all(n1);
  std::iota(all.begin(), all.end(), 0);
  nd.run(std::move(all));

  f.perm.assign(nf, -1);
  f.pos.assign(n, -1);
  for (int k = 0; k < n1; ++k) f.perm[k] = x1v[nd.order[k]];
  for (int k = 0; k < n2; ++k) f.perm[n1 + k] = x2v[k];
  for (int k = 0; k < nf; ++k) f.pos[f.perm[k]] = k;

  // ---- K in solver positions (CSR), couplings, kappa ----------------------
  f.k_ptr.assign(nf + 1, 0);
  f.k_col.clear(); f.k_val.clear();
  double diag_sum = 0.0;
  for (int p = 0; p < nf; ++p) {
    std::vector<std::pair<int, double>> r;
    for (auto& e : rowsK[f.perm[p]])
      if (f.pos[e.first] >= 0) r.push_back({f.pos[e.first], e.second});
    std::sort(r.begin(), r.end(), [](auto& a, auto& b) { return a.first < b.first; });
    for (auto& e : r) {
      f.k_col.push_back(e.first);
      f.k_val.push_back(e.second);
      if (e.first == p) diag_sum += e.second;
    }
    f.k_ptr[p + 1] = (int)f.k_col.size();
  }
  f.kappa_auto = diag_sum / nf;
  f.k12_ptr.assign(n1 + 1, 0); f.k12_col.clear(); f.k12_val.clear();
  for (int p = 0; p < n1; ++p) {
    for (int e = f.k_ptr[p]; e < f.k_ptr[p + 1]; ++e)
      if (f.k_col[e] >= n1) { f.k12_col.push_back(f.k_col[e] - n1); f.k12_val.push_back(f.k_val[e]); }
    f.k12_ptr[p + 1] = (int)f.k12_col.size();
  }
  f.k21_ptr.assign(n2 + 1, 0); f.k21_col.clear(); f.k21_val.clear();
  for (int q = 0; q < n2; ++q) {
    int p = n1 + q;
    for (int e = f.k_ptr[p]; e < f.k_ptr[p + 1]; ++e)
      if (f.k_col[e] < n1) { f.k21_col.push_back(f.k_col[e]); f.k21_val.push_back(f.k_val[e]); }
    f.k21_ptr[q + 1] = (int)f.k21_col.size();
  }

  // ---- supernodes = ND blocks; symbolic structure ---------------------------
  const int nb = (int)nd.blk_begin.size();
  // blocks are created in post-order (children before parents)
  std::vector<std::vector<int>> children(nb);
  for (int b = 0; b < nb; ++b)
    if (nd.blk_parent[b] >= 0) children[nd.blk_parent[b]].push_back(b);
  std::vector<std::vector<int>> R(nb);      // off-diagonal rows (x1 and x2)
  std::vector<int> level(nb, 0);
  std::vector<int> mark(nf, -1);
  for (int b = 0; b < nb; ++b) {
    const int c0 = nd.blk_begin[b], c1 = nd.blk_end[b];
    std::vector<int> r;
    for (int p = c0; p < c1; ++p)
      for (int e = f.k_ptr[p]; e < f.k_ptr[p + 1]; ++e) {
        int q = f.k_col[e];
        if (q >= c1 && mark[q] != b) { mark[q] = b; r.push_back(q); }
      }
    for (int c : children[b]) {
      level[b] = std::max(level[b], level[c] + 1);
      for (int q : R[c])
        if (q >= c1 && mark[q] != b) { mark[q] = b; r.push_back(q); }
    }
    std::sort(r.begin(), r.end());
    R[b] = std::move(r);
  }

  // ---- numeric multifrontal factorisation ----------------------------------
  f.sn.assign(nb, Supernode());
  f.rows.clear();
  f.Z.clear();
  std::vector<std::vector<double>> U(nb);   // update matrices (|R| x |R|, row-major)
  std::vector<double> S(size_t(n2) * n2, 0.0);   // Schur complement accumulator
  std::vector<int> locf(nf, -1);
  int64_t nnz = 0;
  for (int b = 0; b < nb; ++b) {
    const int c0 = nd.blk_begin[b], c1 = nd.blk_end[b], ns = c1 - c0;
    const std::vector<int>& Rb = R[b];
    const int nr = (int)Rb.size(), m = ns + nr;
    for (int k = 0; k < ns; ++k) locf[c0 + k] = k;
    for (int k = 0; k < nr; ++k) locf[Rb[k]] = ns + k;
    std::vector<double> F((size_t)m * m, 0.0);
    for (int p = c0; p < c1; ++p) {
      int lc = p - c0;
      for (int e = f.k_ptr[p]; e < f.k_ptr[p + 1]; ++e) {
        int q = f.k_col[e];
        if (q >= p) F[(size_t)locf[q] * m + lc] += f.k_val[e];
      }
    }
    for (int c : children[b]) {
      const std::vector<int>& Rc = R[c];
      const std::vector<double>& Uc = U[c];
      const int nc = (int)Rc.size();
      for (int i = 0; i < nc; ++i) {
        const int li = locf[Rc[i]];
        for (int j = 0; j <= i; ++j) F[(size_t)li * m + locf[Rc[j]]] += Uc[(size_t)i * nc + j];
      }
      std::vector<double>().swap(U[c]);
    }
    if (!potrf_lower(F.data(), ns, m)) return FSIM_ENOT_SPD;
    double* Fd = F.data();
    parallel_for(nr, [&](int64_t a, int64_t e) {
      trsm_rows(Fd, m, ns + (int)a, ns + (int)e, Fd, m, ns);
    });
    // update matrix U_b = F22 - L21 L21^T (lower)
    std::vector<double>& Ub = U[b];
    Ub.assign((size_t)nr * nr, 0.0);
    double* Up = Ub.data();
    parallel_for(nr, [&](int64_t a, int64_t e) {
      for (int64_t i = a; i < e; ++i) {
        const double* li = Fd + (size_t)(ns + i) * m;
        for (int64_t j = 0; j <= i; ++j) {
          const double* lj = Fd + (size_t)(ns + j) * m;
          Up[i * nr + j] = li[ns + j] - dot(li, lj, ns);
        }
      }
    });
    // rows of L_RJ inside x1 come first (R sorted, x2 positions >= n1); the
    // x2 rows are the block H21 L1^-T of Eq. 8 and are kept as well, so that
    // one forward pass yields y2 = r2 - L21 L1^-1 r1 and one backward pass
    // consumes dx2
    int nr1 = 0;
    while (nr1 < nr && Rb[nr1] < n1) ++nr1;
    Supernode& s = f.sn[b];
    s.c0 = c0; s.ns = ns; s.nr1 = nr1; s.nr = nr; s.level = level[b];
    s.rows_off = (int64_t)f.rows.size();
    for (int k = 0; k < nr; ++k) f.rows.push_back(Rb[k]);
    s.z_off = (int64_t)f.Z.size();
    const int ld = ns + nr;
    f.Z.resize(f.Z.size() + (size_t)ld * ns, 0.0);
    std::vector<double> Li((size_t)ns * ns);
    trtri_lower(Fd, m, ns, Li.data());
    double* Z = f.Z.data() + s.z_off;
    for (int r = 0; r < ns; ++r)
      for (int c = 0; c <= r; ++c) Z[(size_t)c * ld + r] = Li[(size_t)r * ns + c];
    parallel_for(nr, [&](int64_t a, int64_t e) {
      for (int64_t i = a; i < e; ++i) {
        const double* li = Fd + (size_t)(ns + i) * m;
        for (int c = 0; c < ns; ++c) {
          double acc = 0.0;
          for (int k = c; k < ns; ++k) acc += li[k] * Li[(size_t)k * ns + c];
          Z[(size_t)c * ld + ns + i] = acc;
        }
      }
    });
    nnz += (int64_t)ns * (ns + 1) / 2 + (int64_t)ns * nr;
    // roots of the x1 forest pass their (x2-only) update into Sigma
    if (nd.blk_parent[b] < 0) {
      for (int i = 0; i < nr; ++i) {
        const int qi = Rb[i] - n1;
        for (int j = 0; j <= i; ++j) {
          const int qj = Rb[j] - n1;
          double v = Up[(size_t)i * nr + j];
          S[(size_t)qi * n2 + qj] += v;
          if (qi != qj) S[(size_t)qj * n2 + qi] += v;
        }
      }
      std::vector<double>().swap(U[b]);
    }
    for (int k = 0; k < ns; ++k) locf[c0 + k] = -1;
    for (int k = 0; k < nr; ++k) locf[Rb[k]] = -1;
  }
  f.factor_nnz = nnz;

  // ---- levels -----------------------------------------------------------------
  int L = 0;
  for (int b = 0; b < nb; ++b) L = std::max(L, level[b] + 1);
  f.n_levels = L;
  f.level_ptr.assign(L + 1, 0);
  for (int b = 0; b < nb; ++b) f.level_ptr[level[b] + 1]++;
  for (int l = 0; l < L; ++l) f.level_ptr[l + 1] += f.level_ptr[l];
  f.level_sn.assign(nb, 0);
  std::vector<int> fill(f.level_ptr.begin(), f.level_ptr.end() - 1);
  for (int b = 0; b < nb; ++b) f.level_sn[fill[level[b]]++] = b;

  // ---- Sigma = K22 - K21 K11^-1 K12 and its inverse (Eq. 9, Sec. 3.2) -------
  if (n2 > 0) {
    for (int q = 0; q < n2; ++q) {
      int p = n1 + q;
      for (int e = f.k_ptr[p]; e < f.k_ptr[p + 1]; ++e)
        if (f.k_col[e] >= n1) S[(size_t)q * n2 + (f.k_col[e] - n1)] += f.k_val[e];
    }
    // accumulated updates were subtracted as F22 - L L^T (U holds F22-LL^T of the
    // children's K entries only), so S already equals the Schur complement.
    f.sigma = S;                                   // Sigma itself (Schur-only step)
    if (!potrf_lower(S.data(), n2, n2)) return FSIM_ENOT_SPD;
    std::vector<double> Li((size_t)n2 * n2);
    // triangular inverse, columns in parallel
    double* Sd = S.data();
    double* Lip = Li.data();
    std::fill(Li.begin(), Li.end(), 0.0);
    parallel_for(n2, [&](int64_t a, int64_t e) {
      for (int64_t j = a; j < e; ++j) {
        Lip[j * n2 + j] = 1.0 / Sd[j * n2 + j];
        for (int64_t i = j + 1; i < n2; ++i) {
          const double* li = Sd + i * n2;
          double s = 0.0;
          for (int64_t k = j; k < i; ++k) s += li[k] * Lip[k * n2 + j];
          Lip[i * n2 + j] = -s / li[i];
        }
      }
    });
    // Sigma^-1 = Li^T Li ; with Ut = Li^T (row i of Ut = column i of Li)
    std::vector<double> Ut((size_t)n2 * n2);
    for (int64_t i = 0; i < n2; ++i)
      for (int64_t k = 0; k < n2; ++k) Ut[i * n2 + k] = Lip[k * n2 + i];
    f.sigma_inv.assign((size_t)n2 * n2, 0.0);
    double* Si = f.sigma_inv.data();
    const double* Up = Ut.data();
    parallel_for(n2, [&](int64_t a, int64_t e) {
      for (int64_t i = a; i < e; ++i)
        for (int64_t j = 0; j <= i; ++j) {
          // entries of column i of Li are non-zero for rows >= i
          double v = dot(Up + i * n2 + i, Up + j * n2 + i, (int)(n2 - i));
          Si[i * n2 + j] = v;
          Si[j * n2 + i] = v;
        }
    });
  }
  return FSIM_OK;
}

}  // namespace fsim
