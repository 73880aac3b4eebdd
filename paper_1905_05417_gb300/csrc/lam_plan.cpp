// Host side of the plan: validation, 1D bases and Gauss rules, element
// structure, (material, angle) configurations, thickness pieces and pair
// classes, and the analytic sizes of the sparsity pattern. No CUDA here.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>

#include "lam_internal.h"

namespace lam {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ---------------------------------------------------------------------------
// Gauss-Legendre rule on [-1, 1] (Section 2.4 uses tensor Gauss rules).
// Newton's method on P_n with P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), started
// from Tricomi's approximation of the roots.
// ---------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 1; i <= (n + 1) / 2; ++i) {
    double th = pi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
    double r = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, pc = r;
      for (int k = 2; k <= n; ++k) {
        double pn = ((2 * k - 1) * r * pc - (k - 1) * pm) / k;
        pm = pc;
        pc = pn;
      }
      dp = n * (r * pc - pm) / (r * r - 1.0);
      double step = pc / dp;
      r -= step;
      if (std::fabs(step) <= 4e-17) {
        // one more evaluation of the derivative at the converged root
        pm = 1.0;
        pc = r;
        for (int k = 2; k <= n; ++k) {
          double pn = ((2 * k - 1) * r * pc - (k - 1) * pm) / k;
          pm = pc;
          pc = pn;
        }
        dp = n * (r * pc - pm) / (r * r - 1.0);
        break;
      }
    }
    double wi = 2.0 / ((1.0 - r * r) * dp * dp);
    x[i - 1] = -r;
    x[n - i] = r;
    w[i - 1] = wi;
    w[n - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// ---------------------------------------------------------------------------
// 1D bases
// ---------------------------------------------------------------------------
static lam_status setup_basis(Basis& B, const lam_basis1d& in, const char* name) {
  if (in.kind != LAM_BSPLINE && in.kind != LAM_LAGRANGE) {
    set_error("%s: unknown basis kind %d", name, in.kind);
    return LAM_ERR_INVALID_ARG;
  }
  if (in.degree < 1 || in.degree > kMaxDegree) {
    set_error("%s: degree %d outside [1, %d]", name, in.degree, kMaxDegree);
    return LAM_ERR_INVALID_ARG;
  }
  if (!in.knots || in.n_knots < 2) {
    set_error("%s: missing knots", name);
    return LAM_ERR_INVALID_ARG;
  }
  B.kind = in.kind;
  B.p = in.degree;
  B.knots.assign(in.knots, in.knots + in.n_knots);
  const int p = B.p;
  const int nk = in.n_knots;
  for (int k = 0; k < nk; ++k)
    if (!std::isfinite(B.knots[k])) {
      set_error("%s: non-finite knot", name);
      return LAM_ERR_INVALID_ARG;
    }
  if (B.kind == LAM_LAGRANGE) {
    for (int k = 0; k + 1 < nk; ++k)
      if (!(B.knots[k] < B.knots[k + 1])) {
        set_error("%s: Lagrange breakpoints must increase strictly", name);
        return LAM_ERR_INVALID_ARG;
      }
    B.nel = nk - 1;
    B.n = p * B.nel + 1;
    for (int e = 0; e < B.nel; ++e) {
      B.ea.push_back(B.knots[e]);
      B.eb.push_back(B.knots[e + 1]);
      B.span.push_back(e);
      B.first.push_back(p * e);
    }
  } else {
    if (nk < 2 * (p + 1)) {
      set_error("%s: knot vector too short for degree %d", name, p);
      return LAM_ERR_INVALID_ARG;
    }
    for (int k = 0; k + 1 < nk; ++k)
      if (B.knots[k + 1] < B.knots[k]) {
        set_error("%s: knots must not decrease", name);
        return LAM_ERR_INVALID_ARG;
      }
    for (int k = 1; k <= p; ++k)
      if (B.knots[k] != B.knots[0] || B.knots[nk - 1 - k] != B.knots[nk - 1]) {
        set_error("%s: knot vector must be open (end knots repeated degree + 1 times)", name);
        return LAM_ERR_INVALID_ARG;
      }
    if (!(B.knots[p] < B.knots[p + 1]) && nk == 2 * (p + 1)) {
      set_error("%s: empty parametric domain", name);
      return LAM_ERR_INVALID_ARG;
    }
    // interior multiplicity <= p
    int run = 1;
    for (int k = p + 1; k < nk - p - 1; ++k) {
      run = (B.knots[k] == B.knots[k - 1] && k - 1 > p) ? run + 1 : 1;
      if (run > p) {
        set_error("%s: interior knot multiplicity exceeds the degree", name);
        return LAM_ERR_INVALID_ARG;
      }
    }
    B.n = nk - p - 1;
    for (int s = p; s <= nk - p - 2; ++s) {
      if (B.knots[s] < B.knots[s + 1]) {
        B.ea.push_back(B.knots[s]);
        B.eb.push_back(B.knots[s + 1]);
        B.span.push_back(s);
        B.first.push_back(s - p);
      }
    }
    B.nel = (int)B.ea.size();
  }
  // supports and neighbour ranges
  B.elo.assign(B.n, -1);
  B.ehi.assign(B.n, -1);
  for (int e = 0; e < B.nel; ++e)
    for (int k = 0; k <= p; ++k) {
      int i = B.first[e] + k;
      if (B.elo[i] < 0) B.elo[i] = e;
      B.ehi[i] = e;
    }
  B.lo.resize(B.n);
  B.len.resize(B.n);
  for (int i = 0; i < B.n; ++i) {
    if (B.elo[i] < 0) {
      set_error("%s: function %d has an empty support", name, i);
      return LAM_ERR_INVALID_ARG;
    }
    B.lo[i] = B.first[B.elo[i]];
    B.len[i] = B.first[B.ehi[i]] + p - B.lo[i] + 1;
  }
  B.colors = 1;
  for (int e = 0; e < B.nel; ++e) {
    int e2 = e;
    while (e2 + 1 < B.nel && B.first[e2 + 1] <= B.first[e] + p) ++e2;
    B.colors = std::max(B.colors, e2 - e + 1);
  }
  return LAM_OK;
}

// Values and derivatives of the p+1 functions of element e at the point
// x_local (measured from the element's left end, so that structurally equal
// elements give equal tables). B-spline: de Boor's triangular scheme on the
// local knot differences; Lagrange: barycentric form on equispaced nodes.
static void eval_basis_local(const Basis& B, int e, double xl, double* val, double* der) {
  const int p = B.p;
  if (B.kind == LAM_BSPLINE) {
    const int s = B.span[e];
    const double ts = B.knots[s];
    double left[kMaxDegree + 2], right[kMaxDegree + 2], N[kMaxDegree + 2];
    double Nm[kMaxDegree + 2];  // degree p-1 values
    N[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
      left[j] = xl - (B.knots[s + 1 - j] - ts);
      right[j] = (B.knots[s + j] - ts) - xl;
      double saved = 0.0;
      for (int r = 0; r < j; ++r) {
        double tmp = N[r] / (right[r + 1] + left[j - r]);
        N[r] = saved + right[r + 1] * tmp;
        saved = left[j - r] * tmp;
      }
      N[j] = saved;
      if (j == p - 1)
        for (int r = 0; r <= j; ++r) Nm[r] = N[r];
    }
    if (p == 1) Nm[0] = 1.0;
    for (int k = 0; k <= p; ++k) val[k] = N[k];
    // dN_{i,p} = p (N_{i,p-1}/(t_{i+p}-t_i) - N_{i+1,p-1}/(t_{i+p+1}-t_{i+1})),
    // i = s-p+k; the degree p-1 functions of span s are i = s-p+1..s (Nm[0..p-1]).
    for (int k = 0; k <= p; ++k) {
      int i = s - p + k;
      double a = (k >= 1) ? Nm[k - 1] : 0.0;  // N_{i,p-1}
      double b = (k <= p - 1) ? Nm[k] : 0.0;   // N_{i+1,p-1}
      double d = 0.0;
      if (a != 0.0) d += a / (B.knots[i + p] - B.knots[i]);
      if (b != 0.0) d -= b / (B.knots[i + p + 1] - B.knots[i + 1]);
      der[k] = p * d;
    }
    return;
  }
  const double h = B.eb[e] - B.ea[e];
  double nodes[kMaxDegree + 1], wb[kMaxDegree + 1];
  for (int k = 0; k <= p; ++k) nodes[k] = h * k / p;
  for (int k = 0; k <= p; ++k) {
    double prod = 1.0;
    for (int m = 0; m <= p; ++m)
      if (m != k) prod *= (nodes[k] - nodes[m]);
    wb[k] = 1.0 / prod;
  }
  int at = -1;
  for (int k = 0; k <= p; ++k)
    if (xl == nodes[k]) at = k;
  if (at >= 0) {
    for (int k = 0; k <= p; ++k) val[k] = (k == at) ? 1.0 : 0.0;
    double sum = 0.0;
    for (int k = 0; k <= p; ++k) {
      if (k == at) continue;
      der[k] = (wb[k] / wb[at]) / (nodes[at] - nodes[k]);
      sum += der[k];
    }
    der[at] = -sum;
    return;
  }
  double denom = 0.0;
  for (int k = 0; k <= p; ++k) denom += wb[k] / (xl - nodes[k]);
  for (int k = 0; k <= p; ++k) {
    val[k] = (wb[k] / (xl - nodes[k])) / denom;
    double s = 0.0;
    for (int m = 0; m <= p; ++m)
      if (m != k) s += 1.0 / (xl - nodes[m]);
    der[k] = val[k] * s;
  }
}

static void build_inplane_table(const Basis& B, const std::vector<double>& gx, const std::vector<double>& gw,
                                std::vector<double>& tab, std::vector<double>& wt) {
  const int nq = (int)gx.size(), p = B.p;
  tab.assign((size_t)B.nel * nq * (p + 1) * 2, 0.0);
  wt.assign((size_t)B.nel * nq, 0.0);
  for (int e = 0; e < B.nel; ++e) {
    const double h = B.eb[e] - B.ea[e];
    for (int q = 0; q < nq; ++q) {
      double val[kMaxDegree + 1], der[kMaxDegree + 1];
      eval_basis_local(B, e, 0.5 * h * (1.0 + gx[q]), val, der);
      for (int k = 0; k <= p; ++k) {
        tab[(((size_t)e * nq + q) * (p + 1) + k) * 2 + 0] = val[k];
        tab[(((size_t)e * nq + q) * (p + 1) + k) * 2 + 1] = der[k];
      }
      wt[(size_t)e * nq + q] = gw[q] * 0.5 * h;
    }
  }
}

// ---------------------------------------------------------------------------
// Configurations: Eq. D for a ply rotated about z, by the Bond stress
// transformation M (sigma_global = M sigma_material): D_global = M D M^T.
// ---------------------------------------------------------------------------
// Bond matrix M(theta) for the Voigt order 11, 22, 33, 12, 13, 23 and its
// derivative in theta (dM may be NULL).
static void bond_matrix(double theta, double* M, double* dM) {
  const double c = std::cos(theta), s = std::sin(theta);
  const double R[3][3] = {{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}};
  const double dR[3][3] = {{-s, -c, 0.0}, {c, -s, 0.0}, {0.0, 0.0, 0.0}};
  static const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
  for (int I = 0; I < 6; ++I) {
    const int a = ii[I], b = jj[I];
    for (int J = 0; J < 6; ++J) {
      const int p = ii[J], q = jj[J];
      M[I * 6 + J] = (J < 3) ? R[a][p] * R[b][q] : R[a][p] * R[b][q] + R[a][q] * R[b][p];
      if (dM)
        dM[I * 6 + J] = (J < 3) ? dR[a][p] * R[b][q] + R[a][p] * dR[b][q]
                                : dR[a][p] * R[b][q] + R[a][p] * dR[b][q] + dR[a][q] * R[b][p] + R[a][q] * dR[b][p];
    }
  }
}

static void material_matrix(const double* C21, double* Dm) {
  int k = 0;
  for (int I = 0; I < 6; ++I)
    for (int J = I; J < 6; ++J) {
      Dm[I * 6 + J] = Dm[J * 6 + I] = C21[k];
      ++k;
    }
}

static void bond_rotate(const double* C21, double theta, double* D) {
  double Dm[36], M[36], T[36];
  material_matrix(C21, Dm);
  bond_matrix(theta, M, nullptr);
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double acc = 0.0;
      for (int K = 0; K < 6; ++K) acc += M[I * 6 + K] * Dm[K * 6 + J];
      T[I * 6 + J] = acc;
    }
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double acc = 0.0;
      for (int K = 0; K < 6; ++K) acc += T[I * 6 + K] * M[J * 6 + K];
      D[I * 6 + J] = acc;
    }
}

static int voigt_index(int i, int j) {
  static const int V[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  return V[i][j];
}

lam_status rebuild_configs(Plan& P) {
  P.cfg_mat.clear();
  P.cfg_angle.clear();
  P.ply_cfg.assign(P.plies.size(), -1);
  for (size_t l = 0; l < P.plies.size(); ++l) {
    int found = -1;
    for (size_t m = 0; m < P.cfg_mat.size(); ++m)
      if (P.cfg_mat[m] == P.plies[l].material && P.cfg_angle[m] == P.plies[l].angle_rad) found = (int)m;
    if (found < 0) {
      found = (int)P.cfg_mat.size();
      P.cfg_mat.push_back(P.plies[l].material);
      P.cfg_angle.push_back(P.plies[l].angle_rad);
    }
    P.ply_cfg[l] = found;
  }
  const int nc = (int)P.cfg_mat.size();
  P.cfgD.assign((size_t)nc * 36, 0.0);
  P.cfgE.assign((size_t)nc * 81, 0.0);
  P.monoclinic = true;
  for (int m = 0; m < nc; ++m) {
    double* D = &P.cfgD[(size_t)m * 36];
    bond_rotate(P.mats[P.cfg_mat[m]].C, P.cfg_angle[m], D);
    for (int I = 0; I < 4; ++I)
      for (int J = 4; J < 6; ++J)
        if (D[I * 6 + J] != 0.0 || D[J * 6 + I] != 0.0) P.monoclinic = false;
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            P.cfgE[(size_t)m * 81 + (c * 3 + d) * 9 + a * 3 + b] = D[voigt_index(c, a) * 6 + voigt_index(d, b)];
  }
  // Appendix A: the bracket C{e_i, e_j}_{pr} = C_{pirj} of every configuration, from the material
  // tensor rotated by R = rot_z(theta) in all four indices (no Bond matrix)
  P.cfgCb.assign((size_t)nc * 81, 0.0);
  for (int m = 0; m < nc; ++m) {
    double Dm[36];
    material_matrix(P.mats[P.cfg_mat[m]].C, Dm);
    double Cm[3][3][3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) Cm[a][b][c][d] = Dm[voigt_index(a, b) * 6 + voigt_index(c, d)];
    const double cs = std::cos(P.cfg_angle[m]), sn = std::sin(P.cfg_angle[m]);
    const double R[3][3] = {{cs, -sn, 0.0}, {sn, cs, 0.0}, {0.0, 0.0, 1.0}};
    double* out = &P.cfgCb[(size_t)m * 81];
    for (int pp = 0; pp < 3; ++pp)
      for (int i = 0; i < 3; ++i)
        for (int r = 0; r < 3; ++r)
          for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c)
                  for (int d = 0; d < 3; ++d) acc += R[pp][a] * R[i][b] * R[r][c] * R[j][d] * Cm[a][b][c][d];
            out[((i * 3 + j) * 3 + pp) * 3 + r] = acc;
          }
  }
  for (auto& pc : P.pieces) pc.cfg = P.ply_cfg[pc.ply];
  const size_t npl = P.plies.size();
  P.ply_M.assign(npl * 36, 0.0);
  P.ply_dM.assign(npl * 36, 0.0);
  P.ply_mat.assign(npl, 0);
  for (size_t l = 0; l < npl; ++l) {
    bond_matrix(P.plies[l].angle_rad, &P.ply_M[l * 36], &P.ply_dM[l * 36]);
    P.ply_mat[l] = P.plies[l].material;
  }
  P.mat_C.assign(P.mats.size() * 36, 0.0);
  for (size_t m = 0; m < P.mats.size(); ++m) material_matrix(P.mats[m].C, &P.mat_C[m * 36]);
  return LAM_OK;
}

// ---------------------------------------------------------------------------
// Adjoint terms: Eq. Q restricted to each ply, for every thickness pair whose
// common support meets the ply, grouped by ply. Geometry only (the plies'
// positions do not change after plan creation).
// ---------------------------------------------------------------------------
static void build_adjoint_terms(Plan& P) {
  const Basis& T = P.t;
  const int nq = P.nqt, q1 = T.p + 1, npl = (int)P.plies.size();
  std::vector<std::vector<std::pair<int, std::array<double, 4>>>> per_ply(npl);
  for (int64_t pr = 0; pr < P.nnz_t; ++pr) {
    const int i = P.tp_row[pr], j = P.tp_col[pr];
    std::vector<std::array<double, 4>> acc(npl, std::array<double, 4>{0.0, 0.0, 0.0, 0.0});
    std::vector<char> hit(npl, 0);
    for (int e = P.tp_e0[pr]; e <= P.tp_e1[pr]; ++e) {
      const int a = i - T.first[e], b = j - T.first[e];
      for (int pc = P.piece_begin[e]; pc < P.piece_begin[e + 1]; ++pc) {
        const int l = P.pieces[pc].ply;
        hit[l] = 1;
        for (int g = 0; g < nq; ++g) {
          const double* tb = &P.tabT[((size_t)pc * nq + g) * q1 * 2];
          const double w = P.wT[(size_t)pc * nq + g];
          acc[l][0] += w * tb[a * 2] * tb[b * 2];
          acc[l][1] += w * tb[a * 2] * tb[b * 2 + 1];
          acc[l][2] += w * tb[a * 2 + 1] * tb[b * 2];
          acc[l][3] += w * tb[a * 2 + 1] * tb[b * 2 + 1];
        }
      }
    }
    for (int l = 0; l < npl; ++l)
      if (hit[l]) per_ply[l].push_back({(int)pr, acc[l]});
  }
  double mx[4] = {0.0, 0.0, 0.0, 0.0};
  for (auto& v : per_ply)
    for (auto& t : v)
      for (int k = 0; k < 4; ++k) mx[k] = std::max(mx[k], std::fabs(t.second[k]));
  for (int k = 0; k < 4; ++k) {
    int e = 0;
    std::frexp(mx[k], &e);  // mx < 2^e
    P.adj_qscale[k] = mx[k] > 0.0 ? std::ldexp(1.0, e) : 1.0;
  }
  P.adj_begin.assign(npl + 1, 0);
  P.adj_pair.clear();
  P.adj_q.clear();
  P.adj_qdf.clear();
  P.adj_max_terms = 0;
  for (int l = 0; l < npl; ++l) {
    P.adj_begin[l] = (int)P.adj_pair.size();
    P.adj_max_terms = std::max(P.adj_max_terms, (int)per_ply[l].size());
    for (auto& t : per_ply[l]) {
      P.adj_pair.push_back(t.first);
      float hi[4], lo[4];
      for (int k = 0; k < 4; ++k) {
        const double q = t.second[k] / P.adj_qscale[k];
        P.adj_q.push_back(q);
        hi[k] = (float)q;
        lo[k] = (float)(q - (double)hi[k]);
      }
      for (int k = 0; k < 4; ++k) P.adj_qdf.push_back(hi[k]);
      for (int k = 0; k < 4; ++k) P.adj_qdf.push_back(lo[k]);
    }
  }
  P.adj_begin[npl] = (int)P.adj_pair.size();
}

// ---------------------------------------------------------------------------
// Thickness pieces (Eq. C_layers per element) and their tables
// ---------------------------------------------------------------------------
static lam_status build_pieces(Plan& P) {
  const Basis& T = P.t;
  P.pieces.clear();
  P.piece_begin.assign(T.nel + 1, 0);
  const double z_start = T.knots.front();
  std::vector<double> tops(P.plies.size());
  double z = z_start;
  for (size_t l = 0; l < P.plies.size(); ++l) {
    z += P.plies[l].thickness;
    tops[l] = z;
  }
  for (int e = 0; e < T.nel; ++e) {
    P.piece_begin[e] = (int)P.pieces.size();
    const double a = T.ea[e], b = T.eb[e], snap = 1e-10 * (b - a);
    std::vector<double> cuts{a};
    for (size_t l = 0; l + 1 < P.plies.size(); ++l)
      if (tops[l] > a + snap && tops[l] < b - snap) cuts.push_back(tops[l]);
    cuts.push_back(b);
    for (size_t k = 0; k + 1 < cuts.size(); ++k) {
      const double mid = 0.5 * (cuts[k] + cuts[k + 1]);
      int ply = (int)P.plies.size() - 1;
      for (size_t l = 0; l < P.plies.size(); ++l)
        if (mid < tops[l]) {
          ply = (int)l;
          break;
        }
      P.pieces.push_back(Piece{e, ply, 0, cuts[k], cuts[k + 1]});
    }
  }
  P.piece_begin[T.nel] = (int)P.pieces.size();
  const int nq = P.nqt, q1 = T.p + 1;
  P.tabT.assign(P.pieces.size() * nq * q1 * 2, 0.0);
  P.wT.assign(P.pieces.size() * nq, 0.0);
  for (size_t pc = 0; pc < P.pieces.size(); ++pc) {
    const Piece& PC = P.pieces[pc];
    const double a = T.ea[PC.elem];
    const double off = PC.z0 - a, h = PC.z1 - PC.z0;
    for (int q = 0; q < nq; ++q) {
      double val[kMaxDegree + 1], der[kMaxDegree + 1];
      eval_basis_local(T, PC.elem, off + 0.5 * h * (1.0 + P.gxt[q]), val, der);
      for (int k = 0; k < q1; ++k) {
        P.tabT[((pc * nq + q) * q1 + k) * 2 + 0] = val[k];
        P.tabT[((pc * nq + q) * q1 + k) * 2 + 1] = der[k];
      }
      P.wT[pc * nq + q] = P.gwt[q] * 0.5 * h;
    }
  }
  return LAM_OK;
}

// ---------------------------------------------------------------------------
// Thickness pairs, their Q vectors (Eq. Q summed per configuration), and the
// classes of equal vectors used by the combine.
// ---------------------------------------------------------------------------
static lam_status build_classes(Plan& P) {
  const Basis& T = P.t;
  const int nc = (int)P.cfg_mat.size(), nq = P.nqt, q1 = T.p + 1;
  const int64_t npairs = P.nnz_t;
  P.host_q.assign((size_t)npairs * nc * 4, 0.0);
  std::vector<std::vector<int>> terms(npairs);
  for (int64_t pr = 0; pr < npairs; ++pr) {
    const int i = P.tp_row[pr], j = P.tp_col[pr];
    double* q = &P.host_q[(size_t)pr * nc * 4];
    for (int e = P.tp_e0[pr]; e <= P.tp_e1[pr]; ++e) {
      const int a = i - T.first[e], b = j - T.first[e];
      for (int pc = P.piece_begin[e]; pc < P.piece_begin[e + 1]; ++pc) {
        const int m = P.pieces[pc].cfg;
        if (std::find(terms[pr].begin(), terms[pr].end(), m) == terms[pr].end()) terms[pr].push_back(m);
        for (int g = 0; g < nq; ++g) {
          const double* tb = &P.tabT[((size_t)pc * nq + g) * q1 * 2];
          const double w = P.wT[(size_t)pc * nq + g];
          const double Ta = tb[a * 2], dTa = tb[a * 2 + 1], Tb = tb[b * 2], dTb = tb[b * 2 + 1];
          q[m * 4 + 0] += w * Ta * Tb;
          q[m * 4 + 1] += w * Ta * dTb;
          q[m * 4 + 2] += w * dTa * Tb;
          q[m * 4 + 3] += w * dTa * dTb;
        }
      }
    }
    std::sort(terms[pr].begin(), terms[pr].end());
  }
  double scale[4] = {0, 0, 0, 0};
  for (size_t k = 0; k < P.host_q.size(); ++k) scale[k % 4] = std::max(scale[k % 4], std::fabs(P.host_q[k]));
  for (int ab = 0; ab < 4; ++ab) P.q_scale[ab] = scale[ab];
  const double tol = P.class_tol;
  std::vector<int> cls_of(npairs, -1);
  std::vector<int> reps;
  for (int64_t pr = 0; pr < npairs; ++pr) {
    const double* q = &P.host_q[(size_t)pr * nc * 4];
    int found = -1;
    for (size_t u = 0; u < reps.size() && found < 0; ++u) {
      const int r = reps[u];
      if (terms[r] != terms[pr]) continue;
      const double* qr = &P.host_q[(size_t)r * nc * 4];
      bool same = true;
      for (int m : terms[pr])
        for (int ab = 0; ab < 4 && same; ++ab) {
          const double d = std::fabs(q[m * 4 + ab] - qr[m * 4 + ab]);
          same = (tol == 0.0) ? (q[m * 4 + ab] == qr[m * 4 + ab]) : (d <= tol * scale[ab]);
        }
      if (same) found = (int)u;
    }
    if (found < 0) {
      found = (int)reps.size();
      reps.push_back((int)pr);
    }
    cls_of[pr] = found;
  }
  P.ncls = (int)reps.size();
  P.cls_rep = reps;
  P.pair_cls = cls_of;
  P.cls_cfgs.assign(P.ncls, {});
  for (int u = 0; u < P.ncls; ++u) P.cls_cfgs[u] = terms[reps[u]];
  P.cls_term_begin.assign(P.ncls + 1, 0);
  P.cls_terms.clear();
  for (int u = 0; u < P.ncls; ++u) {
    P.cls_term_begin[u] = (int)P.cls_terms.size();
    for (int m : terms[reps[u]]) P.cls_terms.push_back(m);
  }
  P.cls_term_begin[P.ncls] = (int)P.cls_terms.size();
  P.cls_occ_begin.assign(P.ncls + 1, 0);
  std::vector<int> count(P.ncls, 0);
  for (int64_t pr = 0; pr < npairs; ++pr) ++count[cls_of[pr]];
  for (int u = 0; u < P.ncls; ++u) P.cls_occ_begin[u + 1] = P.cls_occ_begin[u] + count[u];
  P.occ_A.assign(npairs, 0);
  P.occ_lt.assign(npairs, 0);
  P.occ_k.assign(npairs, 0);
  P.occ_it.assign(npairs, 0);
  std::vector<int> fill(P.cls_occ_begin.begin(), P.cls_occ_begin.end() - 1);
  for (int64_t pr = 0; pr < npairs; ++pr) {
    const int u = cls_of[pr], o = fill[u]++;
    const int i = P.tp_row[pr];
    P.occ_A[o] = 9 * P.LTb[i] * P.nnz_s;
    P.occ_lt[o] = T.len[i];
    P.occ_k[o] = P.tp_col[pr] - T.lo[i];
    P.occ_it[o] = i;
  }
  return LAM_OK;
}

// ---------------------------------------------------------------------------
// Thickness chunks of the streaming combine: consecutive thickness rows whose
// pairs use at most kc_slots distinct classes (the slices of one in-plane row
// that fit in shared memory). A uniform stack is one chunk; uneven plies, where
// almost every pair is its own class, give chunks of a few plies.
// ---------------------------------------------------------------------------
// Two classes agree on the Q terms (a, b) of one kind: the same configurations,
// and those Q values equal (to class_tol of the largest |Q| of the same term).
static bool same_q_kind(const Plan& P, int cu, int cv, int a, int b) {
  if (P.cls_cfgs[cu] != P.cls_cfgs[cv]) return false;
  const int nc = (int)P.cfg_mat.size();
  const double* qu = &P.host_q[(size_t)P.cls_rep[cu] * nc * 4];
  const double* qv = &P.host_q[(size_t)P.cls_rep[cv] * nc * 4];
  for (int m : P.cls_cfgs[cu])
    for (int ab : {a, b}) {
      const double x = qu[m * 4 + ab], y = qv[m * 4 + ab];
      if (P.class_tol == 0.0 ? x != y : std::fabs(x - y) > P.class_tol * P.q_scale[ab]) return false;
    }
  return true;
}

static void build_chunks_with(Plan& P, int slots) {
  P.ck_it.clear();
  P.ck_term.clear();
  P.ck_nslot.clear();
  P.ckt_slot.clear();
  P.ckt_cfg.clear();
  P.ckt_rep.clear();
  P.ckt_first.clear();
  P.ck_sterm.clear();
  P.ck_nblk.clear();
  P.cks_slot.clear();
  P.cks_cfg.clear();
  P.cks_rep.clear();
  P.cks_first.clear();
  P.ck_copy.clear();
  P.ckc_dst.clear();
  P.ckc_src.clear();
  P.pair_slot.assign(P.nnz_t, 0);
  P.kc_slots = slots;
  std::vector<int> slot_of(P.ncls, -1), members;
  auto close = [&](int it1) {
    // terms of the chunk's classes, sorted by configuration
    const int t0 = (int)P.ckt_slot.size();
    std::vector<std::array<int, 3>> tm;  // (cfg, slot, class)
    for (int u : members)
      for (int m : P.cls_cfgs[u]) tm.push_back({m, slot_of[u], u});
    std::stable_sort(tm.begin(), tm.end(), [](const std::array<int, 3>& x, const std::array<int, 3>& y) {
      return x[0] < y[0];
    });
    std::vector<char> seen(members.size(), 0);
    for (auto& t : tm) {
      P.ckt_cfg.push_back(t[0]);
      P.ckt_slot.push_back(t[1]);
      P.ckt_rep.push_back(P.cls_rep[t[2]]);
      P.ckt_first.push_back(seen[t[1]] ? 0 : 1);
      seen[t[1]] = 1;
    }
    P.ck_term.push_back(t0);
    P.ck_nslot.push_back((int)members.size());
    // Monoclinic plates: an entry (c, d) with c, d both in-plane or both z meets
    // Q_11 and Q_22 only (its "block" kind), the others Q_12 and Q_21 only ("off"
    // kind). Slots whose classes agree on a kind's Q terms have equal slices for
    // that kind's entries: only the first of them (its source) is computed, the
    // others are copied from it. (Q_11, Q_22 are symmetric in the thickness pair,
    // so mirror pairs share their block slices; Q_12, Q_21 of a pair inside one
    // element do not depend on the element's thickness, so same-type pairs of
    // plies of one configuration share their off slices.)
    const int ns_ = (int)members.size();
    std::vector<int> src_b(ns_), src_o(ns_);
    for (int u = 0; u < ns_; ++u) {
      src_b[u] = src_o[u] = u;
      for (int v = 0; v < u && src_b[u] == u; ++v)
        if (src_b[v] == v && same_q_kind(P, members[v], members[u], 0, 3)) src_b[u] = v;
      for (int v = 0; v < u && src_o[u] == u; ++v)
        if (src_o[v] == v && same_q_kind(P, members[v], members[u], 1, 2)) src_o[u] = v;
    }
    P.ck_sterm.push_back((int)P.cks_slot.size());
    P.ck_copy.push_back((int)P.ckc_dst.size());
    for (int kind = 0; kind < 2; ++kind) {
      const std::vector<int>& src = kind == 0 ? src_b : src_o;
      std::vector<char> seen2(ns_, 0);
      int n = 0;
      for (auto& t : tm)  // already sorted by configuration
        if (src[t[1]] == t[1]) {
          P.cks_cfg.push_back(t[0]);
          P.cks_slot.push_back(t[1]);
          P.cks_rep.push_back(P.cls_rep[t[2]]);
          P.cks_first.push_back(seen2[t[1]] ? 0 : 1);
          seen2[t[1]] = 1;
          ++n;
        }
      if (kind == 0) P.ck_nblk.push_back(n);
      for (int u = 0; u < ns_; ++u)
        if (src[u] != u) {
          P.ckc_dst.push_back(2 * u + kind);
          P.ckc_src.push_back(src[u]);
        }
    }
    (void)it1;
    for (int u : members) slot_of[u] = -1;
    members.clear();
  };
  P.ck_it.push_back(0);
  for (int it = 0; it < (int)P.nt; ++it) {
    int fresh = 0;
    std::vector<int> row;
    for (int64_t pr = P.LTb[it]; pr < P.LTb[it + 1]; ++pr) {
      const int u = P.pair_cls[pr];
      if (slot_of[u] < 0 && std::find(row.begin(), row.end(), u) == row.end()) {
        row.push_back(u);
        ++fresh;
      }
    }
    if ((int)members.size() + fresh > P.kc_slots) {
      close(it);
      P.ck_it.push_back(it);
    }
    for (int64_t pr = P.LTb[it]; pr < P.LTb[it + 1]; ++pr) {
      const int u = P.pair_cls[pr];
      if (slot_of[u] < 0) {
        slot_of[u] = (int)members.size();
        members.push_back(u);
      }
      P.pair_slot[pr] = slot_of[u];
    }
  }
  close((int)P.nt);
  P.ck_it.push_back((int)P.nt);
  P.ck_term.push_back((int)P.ckt_slot.size());
  P.ck_sterm.push_back((int)P.cks_slot.size());
  P.ck_copy.push_back((int)P.ckc_dst.size());
}

void build_chunks(Plan& P) {
  int max_lt = 1;
  for (int v : P.t.len) max_lt = std::max(max_lt, v);
  const size_t stride_bytes = (size_t)kcs_stride(P) * sizeof(double);
  const size_t budget = kcs_budget(P);
  int slots = (int)(budget / stride_bytes);
  if (9 * max_len_s(P) <= 512) {
    // fewer slots (more chunks) until the CTAs an SM can hold by registers fit
    // by shared memory too; at least one thickness row per chunk
    for (; slots >= max_lt; --slots) {
      build_chunks_with(P, slots);
      if (kcs_smem(P) <= budget) return;
    }
    build_chunks_with(P, max_lt);
    if (kcs_smem(P) <= 200 * 1024) return;
  }
  // class-major combine
  P.kc_slots = 0;
  P.ck_it.clear();
  P.ck_term.clear();
  P.ck_nslot.clear();
  P.ckt_slot.clear();
  P.ckt_cfg.clear();
  P.ckt_rep.clear();
  P.ckt_first.clear();
  P.ck_sterm.clear();
  P.ck_nblk.clear();
  P.cks_slot.clear();
  P.cks_cfg.clear();
  P.cks_rep.clear();
  P.cks_first.clear();
  P.ck_copy.clear();
  P.ckc_dst.clear();
  P.ckc_src.clear();
  P.pair_slot.assign(P.nnz_t, 0);
}

static void build_colourings(Plan& P) {
  const int cu = P.u.colors, cv = P.v.colors, ct = P.t.colors;
  const int nc2 = cu * cv, nc3 = cu * cv * ct;
  std::vector<std::vector<int>> c2(nc2), c3(nc3);
  for (int ey = 0; ey < P.v.nel; ++ey)
    for (int ex = 0; ex < P.u.nel; ++ex) c2[(ex % cu) + cu * (ey % cv)].push_back(ey * P.u.nel + ex);
  for (int et = 0; et < P.t.nel; ++et)
    for (int ey = 0; ey < P.v.nel; ++ey)
      for (int ex = 0; ex < P.u.nel; ++ex)
        c3[(ex % cu) + cu * ((ey % cv) + cv * (et % ct))].push_back((et * P.v.nel + ey) * P.u.nel + ex);
  P.col2_begin.assign(nc2 + 1, 0);
  P.col2_elem.clear();
  for (int c = 0; c < nc2; ++c) {
    P.col2_begin[c] = (int)P.col2_elem.size();
    P.col2_elem.insert(P.col2_elem.end(), c2[c].begin(), c2[c].end());
  }
  P.col2_begin[nc2] = (int)P.col2_elem.size();
  P.col3_begin.assign(nc3 + 1, 0);
  P.col3_elem.clear();
  for (int c = 0; c < nc3; ++c) {
    P.col3_begin[c] = (int)P.col3_elem.size();
    P.col3_elem.insert(P.col3_elem.end(), c3[c].begin(), c3[c].end());
  }
  P.col3_begin[nc3] = (int)P.col3_elem.size();
}

lam_status build_plan(Plan& P, const lam_inplane* inplane, const lam_basis1d* thickness, const lam_ply* plies,
                      int32_t n_plies, const lam_material* materials, int32_t n_materials, const lam_options* opt) {
  if (!inplane || !thickness || !plies || !materials) {
    set_error("lam_plan_create: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam_status st;
  if ((st = setup_basis(P.u, inplane->u, "in-plane u")) != LAM_OK) return st;
  if ((st = setup_basis(P.v, inplane->v, "in-plane v")) != LAM_OK) return st;
  if ((st = setup_basis(P.t, *thickness, "thickness")) != LAM_OK) return st;
  if (P.u.kind != P.v.kind) {
    set_error("in-plane u and v must use the same basis kind");
    return LAM_ERR_INVALID_ARG;
  }
  if (!inplane->ctrl) {
    set_error("in-plane control points missing");
    return LAM_ERR_INVALID_ARG;
  }
  P.ns = (int64_t)P.u.n * P.v.n;
  P.nt = P.t.n;
  P.n_dof = 3 * P.ns * P.nt;
  if (P.n_dof > std::numeric_limits<int32_t>::max()) {
    set_error("n_dof %lld exceeds the int32 column index range", (long long)P.n_dof);
    return LAM_ERR_UNSUPPORTED;
  }
  const int cdim = inplane->ctrl_dim == 0 ? 2 : inplane->ctrl_dim;
  if (cdim != 2 && cdim != 3) {
    set_error("ctrl_dim must be 2 or 3 (got %d)", inplane->ctrl_dim);
    return LAM_ERR_INVALID_ARG;
  }
  for (int64_t k = 0; k < cdim * P.ns; ++k)
    if (!std::isfinite(inplane->ctrl[k])) {
      set_error("non-finite control point");
      return LAM_ERR_INVALID_ARG;
    }
  const double* ex = inplane->extrusion;
  if (!std::isfinite(ex[0]) || !std::isfinite(ex[1]) || !std::isfinite(ex[2])) {
    set_error("non-finite extrusion direction");
    return LAM_ERR_INVALID_ARG;
  }
  const bool ez = (ex[0] == 0.0 && ex[1] == 0.0 && (ex[2] == 0.0 || ex[2] == 1.0));
  P.shell = cdim == 3 || !ez;
  if (ex[0] != 0.0 || ex[1] != 0.0 || ex[2] != 0.0) {
    P.extrusion[0] = ex[0];
    P.extrusion[1] = ex[1];
    P.extrusion[2] = ex[2];
  }
  P.ctrl.resize(2 * P.ns);
  P.ctrl3.clear();
  if (P.shell) P.ctrl3.resize(3 * P.ns);
  for (int64_t i = 0; i < P.ns; ++i) {
    P.ctrl[2 * i] = inplane->ctrl[cdim * i];
    P.ctrl[2 * i + 1] = inplane->ctrl[cdim * i + 1];
    if (P.shell) {
      P.ctrl3[3 * i] = inplane->ctrl[cdim * i];
      P.ctrl3[3 * i + 1] = inplane->ctrl[cdim * i + 1];
      P.ctrl3[3 * i + 2] = cdim == 3 ? inplane->ctrl[cdim * i + 2] : 0.0;
    }
  }
  P.weights.clear();
  if (inplane->weights) {
    if (P.u.kind != LAM_BSPLINE) {
      set_error("weights are only accepted with a B-spline (NURBS) in-plane basis");
      return LAM_ERR_INVALID_ARG;
    }
    P.weights.assign(inplane->weights, inplane->weights + P.ns);
    for (double w : P.weights)
      if (!(w > 0.0) || !std::isfinite(w)) {
        set_error("NURBS weights must be positive");
        return LAM_ERR_INVALID_ARG;
      }
  }
  if (n_plies < 1 || n_materials < 1) {
    set_error("need at least one ply and one material");
    return LAM_ERR_INVALID_ARG;
  }
  P.plies.assign(plies, plies + n_plies);
  P.mats.assign(materials, materials + n_materials);
  double H = P.t.knots.back() - P.t.knots.front(), sum = 0.0;
  for (int l = 0; l < n_plies; ++l) {
    if (!(P.plies[l].thickness > 0.0) || !std::isfinite(P.plies[l].thickness) ||
        !std::isfinite(P.plies[l].angle_rad) || P.plies[l].material < 0 || P.plies[l].material >= n_materials) {
      set_error("ply %d: invalid thickness, angle or material", l);
      return LAM_ERR_INVALID_ARG;
    }
    sum += P.plies[l].thickness;
  }
  if (std::fabs(sum - H) > 1e-10 * H) {
    set_error("ply thicknesses add up to %.17g, the thickness knots span %.17g", sum, H);
    return LAM_ERR_INVALID_ARG;
  }
  for (int m = 0; m < n_materials; ++m)
    for (int k = 0; k < 21; ++k)
      if (!std::isfinite(P.mats[m].C[k])) {
        set_error("material %d: non-finite constant", m);
        return LAM_ERR_INVALID_ARG;
      }
  lam_options o{0, 0, 0, -1.0, LAM_ARITH_FP64};
  if (opt) o = *opt;
  if (o.arith != LAM_ARITH_FP64 && o.arith != LAM_ARITH_DOUBLE_FLOAT) {
    set_error("unknown arithmetic %d (LAM_ARITH_FP64 or LAM_ARITH_DOUBLE_FLOAT)", (int)o.arith);
    return LAM_ERR_INVALID_ARG;
  }
  P.arith = o.arith;
  P.nqu = o.nq_u > 0 ? o.nq_u : P.u.p + 1;
  P.nqv = o.nq_v > 0 ? o.nq_v : P.v.p + 1;
  P.nqt = o.nq_t > 0 ? o.nq_t : P.t.p + 1;
  if (P.nqu > 16 || P.nqv > 16 || P.nqt > 16) {
    set_error("at most 16 Gauss points per direction");
    return LAM_ERR_UNSUPPORTED;
  }
  if ((P.u.p + 1) * (P.v.p + 1) > 64 || P.nqu * P.nqv > 256) {
    set_error("in-plane element too large for the kernels");
    return LAM_ERR_UNSUPPORTED;
  }
  P.class_tol = o.class_tol < 0.0 ? 1e-13 : o.class_tol;
  gauss_legendre(P.nqu, P.gxu, P.gwu);
  gauss_legendre(P.nqv, P.gxv, P.gwv);
  gauss_legendre(P.nqt, P.gxt, P.gwt);
  build_inplane_table(P.u, P.gxu, P.gwu, P.tabU, P.wU);
  build_inplane_table(P.v, P.gxv, P.gwv, P.tabV, P.wV);
  if ((st = build_pieces(P)) != LAM_OK) return st;
  if ((st = rebuild_configs(P)) != LAM_OK) return st;
  // in-plane pattern: i_s = iy * nx + ix, neighbours (jy major, jx minor)
  P.LSb.assign(P.ns + 1, 0);
  for (int64_t is = 0; is < P.ns; ++is) {
    const int ix = (int)(is % P.u.n), iy = (int)(is / P.u.n);
    P.LSb[is + 1] = P.LSb[is] + (int64_t)P.u.len[ix] * P.v.len[iy];
  }
  P.nnz_s = P.LSb[P.ns];
  P.LTb.assign(P.nt + 1, 0);
  P.tp_row.clear();
  P.tp_col.clear();
  P.tp_e0.clear();
  P.tp_e1.clear();
  for (int it = 0; it < P.nt; ++it) {
    P.LTb[it + 1] = P.LTb[it] + P.t.len[it];
    for (int k = 0; k < P.t.len[it]; ++k) {
      const int jt = P.t.lo[it] + k;
      P.tp_row.push_back(it);
      P.tp_col.push_back(jt);
      P.tp_e0.push_back(std::max(P.t.elo[it], P.t.elo[jt]));
      P.tp_e1.push_back(std::min(P.t.ehi[it], P.t.ehi[jt]));
    }
  }
  P.nnz_t = P.LTb[P.nt];
  P.nnz = 9 * P.nnz_s * P.nnz_t;
  P.tp_A.resize(P.nnz_t);
  P.tp_lt.resize(P.nnz_t);
  P.tp_k.resize(P.nnz_t);
  for (int64_t pr = 0; pr < P.nnz_t; ++pr) {
    const int it = P.tp_row[pr];
    P.tp_A[pr] = 9 * P.LTb[it] * P.nnz_s;
    P.tp_lt[pr] = P.t.len[it];
    P.tp_k[pr] = P.tp_col[pr] - P.t.lo[it];
  }
  if ((st = build_classes(P)) != LAM_OK) return st;
  build_chunks(P);
  build_adjoint_terms(P);
  build_colourings(P);
  return LAM_OK;
}

}  // namespace lam

// ---------------------------------------------------------------------------
// Host-only C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* lam_last_error(void) { return lam::g_err; }

const char* lam_version(void) { return "lam 0.1 (sm_103a, FP64)"; }

lam_status lam_plan_create(lam_plan** out, const lam_inplane* inplane, const lam_basis1d* thickness,
                           const lam_ply* plies, int32_t n_plies, const lam_material* materials,
                           int32_t n_materials, const lam_options* options) {
  if (!out) {
    lam::set_error("lam_plan_create: out is NULL");
    return LAM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  lam_plan* plan = new (std::nothrow) lam_plan();
  if (!plan) {
    lam::set_error("lam_plan_create: out of host memory");
    return LAM_ERR_OOM;
  }
  lam_status st;
  try {
    st = lam::build_plan(plan->p, inplane, thickness, plies, n_plies, materials, n_materials, options);
  } catch (const std::bad_alloc&) {
    lam::set_error("lam_plan_create: out of host memory");
    st = LAM_ERR_OOM;
  }
  if (st != LAM_OK) {
    delete plan;
    return st;
  }
  lam::set_error("");
  *out = plan;
  return LAM_OK;
}

lam_status lam_plan_get_info(const lam_plan* plan, lam_plan_info* info) {
  if (!plan || !info) {
    lam::set_error("lam_plan_get_info: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  const lam::Plan& P = plan->p;
  info->n_dof = P.n_dof;
  info->nnz = P.nnz;
  info->n_s = P.ns;
  info->n_t = P.nt;
  info->nnz_inplane = P.nnz_s;
  info->nnz_thickness = P.nnz_t;
  info->n_configs = (int32_t)P.cfg_mat.size();
  info->n_classes = P.ncls;
  info->monoclinic = P.monoclinic ? 1 : 0;
  info->n_pieces = (int32_t)P.pieces.size();
  info->combine_streaming = lam::use_stream(P) ? 1 : 0;
  info->combine_chunks = (int32_t)P.ck_nslot.size();
  info->shell = P.shell ? 1 : 0;
  info->arith = P.arith;
  info->combine_terms = (int32_t)P.ckt_slot.size();
  info->combine_source_terms = (int32_t)P.cks_slot.size();
  int64_t nblk = 0;
  for (int v : P.ck_nblk) nblk += v;
  info->combine_block_terms = (int32_t)nblk;
  return LAM_OK;
}

lam_status lam_plan_update(lam_plan* plan, const double* ply_angle_rad, int32_t n_plies,
                           const lam_material* materials, int32_t n_materials) {
  if (!plan) {
    lam::set_error("lam_plan_update: plan is NULL");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  if (ply_angle_rad) {
    if (n_plies != (int32_t)P.plies.size()) {
      lam::set_error("lam_plan_update: %d angles for %d plies", n_plies, (int)P.plies.size());
      return LAM_ERR_INVALID_ARG;
    }
    for (int l = 0; l < n_plies; ++l)
      if (!std::isfinite(ply_angle_rad[l])) {
        lam::set_error("lam_plan_update: non-finite angle");
        return LAM_ERR_INVALID_ARG;
      }
  }
  if (materials && n_materials != (int32_t)P.mats.size()) {
    lam::set_error("lam_plan_update: %d materials for %d", n_materials, (int)P.mats.size());
    return LAM_ERR_INVALID_ARG;
  }
  if (ply_angle_rad)
    for (int l = 0; l < n_plies; ++l) P.plies[l].angle_rad = ply_angle_rad[l];
  if (materials) P.mats.assign(materials, materials + n_materials);
  lam::rebuild_configs(P);
  lam::build_classes(P);
  lam::build_chunks(P);
  P.cfg_dirty = true;
  ++P.cfg_version;  // configuration tables are re-uploaded by the next device call
  return LAM_OK;
}

}  // extern "C"
