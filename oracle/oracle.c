/*
 * CPU oracle: plain FP64 stiffness assembly of an extruded layered solid.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Slow on purpose: every quantity is
 * evaluated from its definition, one basis function and one quadrature point at
 * a time, with no blocking, fusion or reordering beyond the formulas below.
 *
 * Paper: P. Antolin, "Fast assembly of Galerkin matrices for 3D solid laminated
 * composites using finite element and isogeometric discretizations" (2019).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - Eq. B_0 / Eq. B_1, third row of B^T: its last entry is read as the second
 *    gradient component (gamma_23 = d2 u3 + d3 u2); shears are engineering
 *    shears, consistent with the Voigt matrix D of Eq. D.
 *  - Eq. Km_1 is read with B^T on the left, as in Eq. K_1 and Eq. P.
 *  - Eq. Q is read as Q_{ab} = int tau_a^{i} tau_b^{j}, tau_1 = T, tau_2 = T',
 *    so that Q_12 = int T^i T'^j pairs with P_12 = int B_1^{iT} D B_2^j.
 *  - The extrusion of Eq. extrusion uses a = e_z and xi^3 = z (physical), so
 *    |DF| is the 2x2 in-plane Jacobian determinant.
 *  - A ply interface closer than 1e-10 of a thickness element's length to one
 *    of its ends is taken to coincide with that end (rounding of cumulative
 *    ply thicknesses must not create sliver pieces).
 *
 * parity unpinned: none of the functions below is unpinned; the pins live in
 * tests/ (closed forms, invariants, library routines, exact rationals).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre quadrature (the tensor Gauss rules of Section 2.4).       */
/* Newton iteration on the Legendre polynomial P_n, evaluated by its        */
/* three-term recurrence; weights w = 2 / ((1 - x^2) P_n'(x)^2).            */
/* ------------------------------------------------------------------------ */
static void legendre_pn(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

int ora_gauss(int32_t n, double* x, double* w) {
  if (n < 1 || n > 64) return -1;
  for (int k = 0; k < n; ++k) {
    double z = cos(ORA_PI * (k + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(n, z, &pn, &dpn);
      double dz = pn / dpn;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    legendre_pn(n, z, &pn, &dpn);
    x[n - 1 - k] = z;
    w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 1D bases (Section 2.2 and the admissible bases listed after Assumption 1)*/
/* ------------------------------------------------------------------------ */
int32_t ora_nfun(const ora_basis1d* b) {
  if (b->kind == ORA_BSPLINE) return b->n_knots - b->degree - 1;
  return b->degree * (b->n_knots - 1) + 1;
}

/* The e-th element: B-spline -> e-th nonempty knot span, Lagrange -> e-th
 * breakpoint interval. Returns the span index (B-spline) or e (Lagrange). */
static int element_of(const ora_basis1d* b, int e, double* a, double* bb, int* first) {
  if (b->kind == ORA_LAGRANGE) {
    if (e < 0 || e >= b->n_knots - 1) return -1;
    *a = b->knots[e];
    *bb = b->knots[e + 1];
    *first = b->degree * e;
    return e;
  }
  int p = b->degree, count = 0;
  for (int s = p; s <= b->n_knots - p - 2; ++s) {
    if (b->knots[s] < b->knots[s + 1]) {
      if (count == e) {
        *a = b->knots[s];
        *bb = b->knots[s + 1];
        *first = s - p;
        return s;
      }
      ++count;
    }
  }
  return -1;
}

int32_t ora_nel(const ora_basis1d* b) {
  if (b->kind == ORA_LAGRANGE) return b->n_knots - 1;
  int p = b->degree, count = 0;
  for (int s = p; s <= b->n_knots - p - 2; ++s)
    if (b->knots[s] < b->knots[s + 1]) ++count;
  return count;
}

/* Cox-de Boor recursion written as its definition: N_{i,0} is the indicator
 * of the span that contains x; N_{i,p} = (x-t_i)/(t_{i+p}-t_i) N_{i,p-1}
 * + (t_{i+p+1}-x)/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}, with 0/0 read as 0. */
static double bs_value(const double* t, int i, int p, int span, double x) {
  if (p == 0) return i == span ? 1.0 : 0.0;
  double v = 0.0;
  double d1 = t[i + p] - t[i];
  double d2 = t[i + p + 1] - t[i + 1];
  if (d1 > 0.0) v += (x - t[i]) / d1 * bs_value(t, i, p - 1, span, x);
  if (d2 > 0.0) v += (t[i + p + 1] - x) / d2 * bs_value(t, i + 1, p - 1, span, x);
  return v;
}

/* dN_{i,p}/dx = p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}. */
static double bs_deriv(const double* t, int i, int p, int span, double x) {
  if (p == 0) return 0.0;
  double v = 0.0;
  double d1 = t[i + p] - t[i];
  double d2 = t[i + p + 1] - t[i + 1];
  if (d1 > 0.0) v += p / d1 * bs_value(t, i, p - 1, span, x);
  if (d2 > 0.0) v -= p / d2 * bs_value(t, i + 1, p - 1, span, x);
  return v;
}

int ora_basis1d_eval(const ora_basis1d* b, int32_t e, double x, double* val, double* der, int32_t* first) {
  double a, bb;
  int f;
  int s = element_of(b, e, &a, &bb, &f);
  if (s < 0 || b->degree < 1) return -1;
  int p = b->degree;
  *first = f;
  if (b->kind == ORA_BSPLINE) {
    for (int k = 0; k <= p; ++k) {
      val[k] = bs_value(b->knots, f + k, p, s, x);
      der[k] = bs_deriv(b->knots, f + k, p, s, x);
    }
    return 0;
  }
  /* Lagrange polynomials on p+1 equispaced nodes of [a, bb]. */
  double nodes[32];
  if (p > 30) return -1;
  for (int k = 0; k <= p; ++k) nodes[k] = a + (bb - a) * k / p;
  for (int k = 0; k <= p; ++k) {
    double v = 1.0;
    for (int m = 0; m <= p; ++m)
      if (m != k) v *= (x - nodes[m]) / (nodes[k] - nodes[m]);
    double d = 0.0;
    for (int j = 0; j <= p; ++j) {
      if (j == k) continue;
      double prod = 1.0 / (nodes[k] - nodes[j]);
      for (int m = 0; m <= p; ++m)
        if (m != k && m != j) prod *= (x - nodes[m]) / (nodes[k] - nodes[m]);
      d += prod;
    }
    val[k] = v;
    der[k] = d;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Material (Eq. D and the per-layer tensors of Eq. C_layers)               */
/* ------------------------------------------------------------------------ */
/* Voigt index of the symmetric index pair (i, j), order 11,22,33,12,13,23. */
static int voigt(int i, int j) {
  if (i == j) return i;
  if ((i == 0 && j == 1) || (i == 1 && j == 0)) return 3;
  if ((i == 0 && j == 2) || (i == 2 && j == 0)) return 4;
  return 5;
}

/* C'_{ijkl} = R_ip R_jq R_kr R_ls C_pqrs with R the rotation by theta about z;
 * with engineering shears the Voigt matrix holds C_{ijkl} directly. */
void ora_rotated_D(const double* C21, double theta, double* D36) {
  double Dm[6][6];
  int k = 0;
  for (int I = 0; I < 6; ++I)
    for (int J = I; J < 6; ++J) {
      Dm[I][J] = C21[k];
      Dm[J][I] = C21[k];
      ++k;
    }
  double c = cos(theta), s = sin(theta);
  double R[3][3] = {{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}};
  static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int I = 0; I < 6; ++I) {
    for (int J = 0; J < 6; ++J) {
      int i = pairs[I][0], j = pairs[I][1], kk = pairs[J][0], l = pairs[J][1];
      double sum = 0.0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
          for (int r = 0; r < 3; ++r)
            for (int t = 0; t < 3; ++t)
              sum += R[i][p] * R[j][q] * R[kk][r] * R[l][t] * Dm[voigt(p, q)][voigt(r, t)];
      D36[I * 6 + J] = sum;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Strain-displacement matrix of Eq. B_1 (6x3), from a gradient g.          */
/* ------------------------------------------------------------------------ */
static void strain_matrix(const double g[3], double B[6][3]) {
  memset(B, 0, sizeof(double) * 18);
  B[0][0] = g[0];                   /* eps_11 */
  B[1][1] = g[1];                   /* eps_22 */
  B[2][2] = g[2];                   /* eps_33 */
  B[3][0] = g[1]; B[3][1] = g[0];   /* gamma_12 */
  B[4][0] = g[2]; B[4][2] = g[0];   /* gamma_13 */
  B[5][1] = g[2]; B[5][2] = g[1];   /* gamma_23 */
}

/* acc[c][d] += w * (Bi^T D Bj)[c][d] */
static void add_btdb(double w, double Bi[6][3], const double* D36, double Bj[6][3], double* acc) {
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) s += Bi[I][c] * D36[I * 6 + J] * Bj[J][d];
      acc[c * 3 + d] += w * s;
    }
}

/* ------------------------------------------------------------------------ */
/* Problem helpers                                                          */
/* ------------------------------------------------------------------------ */
static int nq_or_default(int nq, int degree) { return nq > 0 ? nq : degree + 1; }

static double thickness_start(const ora_problem* pr) { return pr->t.knots[0]; }

/* Ply pieces of thickness element et: pieces [z0, z1] with the ply that
 * contains their midpoint (Eq. C_layers: one material per layer). */
static int ply_pieces(const ora_problem* pr, int et, double* z0, double* z1, int* ply, int max_pieces) {
  double a, b;
  int first;
  if (element_of(&pr->t, et, &a, &b, &first) < 0) return -1;
  double snap = 1e-10 * (b - a);
  int n = 0;
  double cuts[4096];
  cuts[n++] = a;
  double z = thickness_start(pr);
  for (int l = 0; l < pr->n_plies - 1; ++l) {
    z += pr->ply_thickness[l];
    if (z > a + snap && z < b - snap) {
      if (n >= 4095) return -1;
      cuts[n++] = z;
    }
  }
  cuts[n++] = b;
  if (n - 1 > max_pieces) return -1;
  for (int k = 0; k + 1 < n; ++k) {
    z0[k] = cuts[k];
    z1[k] = cuts[k + 1];
    double mid = 0.5 * (cuts[k] + cuts[k + 1]);
    double top = thickness_start(pr);
    int l = 0;
    for (l = 0; l < pr->n_plies; ++l) {
      top += pr->ply_thickness[l];
      if (mid < top) break;
    }
    if (l >= pr->n_plies) l = pr->n_plies - 1;
    ply[k] = l;
  }
  return n - 1;
}

static int check_problem(const ora_problem* pr) {
  if (pr->u.degree < 1 || pr->v.degree < 1 || pr->t.degree < 1) return -1;
  if (pr->n_plies < 1 || pr->n_materials < 1) return -1;
  double H = pr->t.knots[pr->t.n_knots - 1] - pr->t.knots[0];
  double sum = 0.0;
  for (int l = 0; l < pr->n_plies; ++l) {
    if (!(pr->ply_thickness[l] > 0.0)) return -1;
    if (pr->ply_material[l] < 0 || pr->ply_material[l] >= pr->n_materials) return -1;
    sum += pr->ply_thickness[l];
  }
  if (fabs(sum - H) > 1e-10 * H) return -1;
  return 0;
}

/* In-plane quantities at one point of in-plane element (ex, ey): values R,
 * the Jacobian determinant |DF| and the pulled-back gradients of Eq. gradient
 * split as in Eq. B_2: the 3D function S^k T has the physical gradient
 *   grad(S^k T) = T g1[k] + T' S^k r3,
 * g1[k] = DF^{-T} (dS^k/dxi1, dS^k/dxi2, 0), r3 = DF^{-T} e_3. For the planar
 * map (S = (x, y, 0), a = e_z) g1[k] = (dS/dx, dS/dy, 0) and r3 = e_3. */
typedef struct {
  int nlx, nly, fx, fy;
  double R[64], g1[64][3];
  double r3[3];
  double detJ;
} inplane_point;

/* A general extrusion: a surface in R^3 or a direction other than e_z. */
static int is_shell(const ora_problem* pr) {
  if (pr->ctrl_dim == 3) return 1;
  if (pr->extrusion && (pr->extrusion[0] != 0.0 || pr->extrusion[1] != 0.0 || pr->extrusion[2] != 1.0)) return 1;
  return 0;
}

static void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Gradient of the 3D function (local in-plane k, thickness value T and
 * derivative dT) at an in-plane point: T g1[k] + (dT R[k]) r3. */
static void grad3(const inplane_point* ip, int k, double T, double dT, double out[3]) {
  const double s = dT * ip->R[k];
  for (int c = 0; c < 3; ++c) out[c] = T * ip->g1[k][c] + s * ip->r3[c];
}

static int eval_inplane(const ora_problem* pr, int ex, int ey, double xi, double eta, inplane_point* ip) {
  double Nu[8], dNu[8], Nv[8], dNv[8];
  int fx, fy;
  if (ora_basis1d_eval(&pr->u, ex, xi, Nu, dNu, &fx) < 0) return -1;
  if (ora_basis1d_eval(&pr->v, ey, eta, Nv, dNv, &fy) < 0) return -1;
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nx = ora_nfun(&pr->u);
  ip->nlx = nlx;
  ip->nly = nly;
  ip->fx = fx;
  ip->fy = fy;
  double N[64], N1[64], N2[64], R1[64], R2[64];
  for (int ly = 0; ly < nly; ++ly)
    for (int lx = 0; lx < nlx; ++lx) {
      int k = ly * nlx + lx;
      N[k] = Nu[lx] * Nv[ly];
      N1[k] = dNu[lx] * Nv[ly];
      N2[k] = Nu[lx] * dNv[ly];
    }
  int nl = nlx * nly;
  if (pr->weights) {
    /* NURBS: R = w N / W, dR = w (dN W - N dW) / W^2 */
    double W = 0.0, W1 = 0.0, W2 = 0.0;
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        int k = ly * nlx + lx;
        double wk = pr->weights[(fy + ly) * nx + (fx + lx)];
        W += wk * N[k];
        W1 += wk * N1[k];
        W2 += wk * N2[k];
      }
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        int k = ly * nlx + lx;
        double wk = pr->weights[(fy + ly) * nx + (fx + lx)];
        ip->R[k] = wk * N[k] / W;
        R1[k] = wk * (N1[k] * W - N[k] * W1) / (W * W);
        R2[k] = wk * (N2[k] * W - N[k] * W2) / (W * W);
      }
  } else {
    for (int k = 0; k < nl; ++k) {
      ip->R[k] = N[k];
      R1[k] = N1[k];
      R2[k] = N2[k];
    }
  }
  if (!is_shell(pr)) {
    /* J[a][k] = d x_a / d xi_k = sum_i dR_i/dxi_k X_i[a] */
    double J[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const int cd = pr->ctrl_dim == 3 ? 3 : 2;
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        int k = ly * nlx + lx;
        const double* X = pr->ctrl + cd * ((fy + ly) * nx + (fx + lx));
        J[0][0] += R1[k] * X[0];
        J[0][1] += R2[k] * X[0];
        J[1][0] += R1[k] * X[1];
        J[1][1] += R2[k] * X[1];
      }
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (det == 0.0) return -1;
    /* Jinv[k][a] = d xi_k / d x_a */
    double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    for (int k = 0; k < nl; ++k) {
      ip->g1[k][0] = Ji[0][0] * R1[k] + Ji[1][0] * R2[k];
      ip->g1[k][1] = Ji[0][1] * R1[k] + Ji[1][1] * R2[k];
      ip->g1[k][2] = 0.0;
    }
    ip->r3[0] = 0.0;
    ip->r3[1] = 0.0;
    ip->r3[2] = 1.0;
    ip->detJ = fabs(det);
    return 0;
  }
  /* Eq. extrusion: DF = [dS/dxi1 | dS/dxi2 | a] (columns A[0], A[1], A[2]).
   * The rows of DF^{-1} are the dual vectors g^k = (A[k+1] x A[k+2]) / det DF,
   * so grad = DF^{-T} grad_xi = sum_k g^k d/dxi_k. */
  double A[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  const int cd = pr->ctrl_dim == 3 ? 3 : 2;
  for (int ly = 0; ly < nly; ++ly)
    for (int lx = 0; lx < nlx; ++lx) {
      int k = ly * nlx + lx;
      const double* X = pr->ctrl + cd * ((fy + ly) * nx + (fx + lx));
      for (int c = 0; c < cd; ++c) {
        A[0][c] += R1[k] * X[c];
        A[1][c] += R2[k] * X[c];
      }
    }
  if (pr->extrusion) {
    A[2][0] = pr->extrusion[0];
    A[2][1] = pr->extrusion[1];
    A[2][2] = pr->extrusion[2];
  } else {
    A[2][2] = 1.0;
  }
  double g[3][3], t[3];
  cross3(A[1], A[2], t);
  double det = A[0][0] * t[0] + A[0][1] * t[1] + A[0][2] * t[2];
  if (det == 0.0) return -1;
  for (int k = 0; k < 3; ++k) {
    cross3(A[(k + 1) % 3], A[(k + 2) % 3], t);
    for (int c = 0; c < 3; ++c) g[k][c] = t[c] / det;
  }
  for (int k = 0; k < nl; ++k)
    for (int c = 0; c < 3; ++c) ip->g1[k][c] = g[0][c] * R1[k] + g[1][c] * R2[k];
  for (int c = 0; c < 3; ++c) ip->r3[c] = g[2][c];
  ip->detJ = fabs(det);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Element stiffness, Section 2.4: Gauss rule per element piece, summing    */
/* B^{iT} D_l B^j |DF| w over the points (Eq. K_2 restricted to the element)*/
/* ------------------------------------------------------------------------ */
int ora_element_stiffness(const ora_problem* pr, int32_t ex, int32_t ey, int32_t et, double* out) {
  if (check_problem(pr) < 0) return -1;
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nlt = pr->t.degree + 1;
  int nls = nlx * nly, nl = nls * nlt;
  if (nls > 64 || nlt > 8) return -1;
  memset(out, 0, sizeof(double) * (size_t)nl * nl * 9);
  double ua, ub, va, vb, ta, tb;
  int f;
  if (element_of(&pr->u, ex, &ua, &ub, &f) < 0) return -1;
  if (element_of(&pr->v, ey, &va, &vb, &f) < 0) return -1;
  if (element_of(&pr->t, et, &ta, &tb, &f) < 0) return -1;
  int nqu = nq_or_default(pr->nq_u, pr->u.degree), nqv = nq_or_default(pr->nq_v, pr->v.degree);
  int nqt = nq_or_default(pr->nq_t, pr->t.degree);
  double xu[64], wu[64], xv[64], wv[64], xt[64], wt[64];
  if (ora_gauss(nqu, xu, wu) < 0 || ora_gauss(nqv, xv, wv) < 0 || ora_gauss(nqt, xt, wt) < 0) return -1;
  double z0[512], z1[512];
  int ply[512];
  int npieces = ply_pieces(pr, et, z0, z1, ply, 512);
  if (npieces < 0) return -1;
  double (*B)[6][3] = malloc(sizeof(double) * 18 * nl);
  if (!B) return -1;
  inplane_point ip;
  for (int pc = 0; pc < npieces; ++pc) {
    int l = ply[pc];
    double D[36];
    ora_rotated_D(pr->C21 + 21 * pr->ply_material[l], pr->ply_angle[l], D);
    for (int a = 0; a < nqu; ++a)
      for (int b = 0; b < nqv; ++b) {
        double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[a]);
        double eta = va + 0.5 * (vb - va) * (1.0 + xv[b]);
        if (eval_inplane(pr, ex, ey, xi, eta, &ip) < 0) { free(B); return -1; }
        for (int g = 0; g < nqt; ++g) {
          double z = z0[pc] + 0.5 * (z1[pc] - z0[pc]) * (1.0 + xt[g]);
          double T[8], dT[8];
          int ft;
          if (ora_basis1d_eval(&pr->t, et, z, T, dT, &ft) < 0) { free(B); return -1; }
          double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * wt[g] * 0.5 * (z1[pc] - z0[pc]) * ip.detJ;
          for (int lt = 0; lt < nlt; ++lt)
            for (int ls = 0; ls < nls; ++ls) {
              double grad[3];
              grad3(&ip, ls, T[lt], dT[lt], grad);
              strain_matrix(grad, B[lt * nls + ls]);
            }
          for (int i = 0; i < nl; ++i)
            for (int j = 0; j < nl; ++j) add_btdb(w, B[i], D, B[j], out + ((size_t)i * nl + j) * 9);
        }
      }
  }
  free(B);
  return nl;
}

/* ------------------------------------------------------------------------ */
/* Sparsity: a 3x3 block for every pair of basis functions whose supports   */
/* share a 3D element, found by marking the functions of every element in   */
/* the support of each row function.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;          /* functions */
  int nel;
  int* first;     /* first function of each element */
  int* elo;       /* first element in the support of each function */
  int* ehi;       /* last element in the support of each function */
} support1d;

static int support_build(const ora_basis1d* b, support1d* s) {
  s->n = ora_nfun(b);
  s->nel = ora_nel(b);
  s->first = malloc(sizeof(int) * s->nel);
  s->elo = malloc(sizeof(int) * s->n);
  s->ehi = malloc(sizeof(int) * s->n);
  if (!s->first || !s->elo || !s->ehi) return -1;
  for (int e = 0; e < s->nel; ++e) {
    double a, bb;
    element_of(b, e, &a, &bb, &s->first[e]);
  }
  for (int i = 0; i < s->n; ++i) {
    s->elo[i] = -1;
    s->ehi[i] = -2;
    for (int e = 0; e < s->nel; ++e) {
      if (s->first[e] <= i && i <= s->first[e] + b->degree) {
        if (s->elo[i] < 0) s->elo[i] = e;
        s->ehi[i] = e;
      }
    }
  }
  return 0;
}

static void support_free(support1d* s) {
  free(s->first);
  free(s->elo);
  free(s->ehi);
}

static int cmp_int64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

typedef struct {
  support1d su, sv, st;
  int64_t nbasis;
  int64_t* bptr;   /* basis-level row pointer (nbasis + 1) */
  int64_t* bcol;   /* basis-level neighbours, sorted */
} pattern;

static void pattern_free(pattern* P) {
  support_free(&P->su);
  support_free(&P->sv);
  support_free(&P->st);
  free(P->bptr);
  free(P->bcol);
}

static int pattern_build(const ora_problem* pr, pattern* P) {
  memset(P, 0, sizeof(*P));
  if (support_build(&pr->u, &P->su) < 0 || support_build(&pr->v, &P->sv) < 0 || support_build(&pr->t, &P->st) < 0)
    return -1;
  int nx = P->su.n, ny = P->sv.n, nt = P->st.n;
  int64_t ns = (int64_t)nx * ny;
  P->nbasis = ns * nt;
  unsigned char* mark = calloc((size_t)P->nbasis, 1);
  int64_t* list = malloc(sizeof(int64_t) * (1 << 20));
  P->bptr = malloc(sizeof(int64_t) * (P->nbasis + 1));
  if (!mark || !list || !P->bptr) return -1;
  int pu = pr->u.degree, pv = pr->v.degree, q = pr->t.degree;
  /* pass 1: counts; pass 2: fill */
  for (int pass = 0; pass < 2; ++pass) {
    int64_t pos = 0;
    for (int64_t i = 0; i < P->nbasis; ++i) {
      int it = (int)(i / ns);
      int64_t is = i % ns;
      int iy = (int)(is / nx), ix = (int)(is % nx);
      int64_t cnt = 0;
      for (int et = P->st.elo[it]; et <= P->st.ehi[it]; ++et)
        for (int ey = P->sv.elo[iy]; ey <= P->sv.ehi[iy]; ++ey)
          for (int ex = P->su.elo[ix]; ex <= P->su.ehi[ix]; ++ex)
            for (int lt = 0; lt <= q; ++lt)
              for (int ly = 0; ly <= pv; ++ly)
                for (int lx = 0; lx <= pu; ++lx) {
                  int64_t j = (int64_t)(P->st.first[et] + lt) * ns + (int64_t)(P->sv.first[ey] + ly) * nx +
                              (P->su.first[ex] + lx);
                  if (!mark[j]) {
                    mark[j] = 1;
                    list[cnt++] = j;
                  }
                }
      for (int64_t k = 0; k < cnt; ++k) mark[list[k]] = 0;
      if (pass == 0) {
        P->bptr[i] = pos;
      } else {
        qsort(list, (size_t)cnt, sizeof(int64_t), cmp_int64);
        memcpy(P->bcol + P->bptr[i], list, sizeof(int64_t) * cnt);
      }
      pos += cnt;
    }
    if (pass == 0) {
      P->bptr[P->nbasis] = pos;
      P->bcol = malloc(sizeof(int64_t) * (pos > 0 ? pos : 1));
      if (!P->bcol) return -1;
    }
  }
  free(mark);
  free(list);
  return 0;
}

int ora_sizes(const ora_problem* pr, int64_t* n_dof, int64_t* nnz) {
  if (check_problem(pr) < 0) return -1;
  pattern P;
  if (pattern_build(pr, &P) < 0) return -1;
  *n_dof = 3 * P.nbasis;
  *nnz = 9 * P.bptr[P.nbasis];
  pattern_free(&P);
  return 0;
}

/* Expand the basis-level pattern into the DOF-level CSR (3x3 blocks). */
static void pattern_to_csr(const pattern* P, int64_t* row_ptr, int32_t* col) {
  for (int64_t i = 0; i < P->nbasis; ++i) {
    int64_t len = P->bptr[i + 1] - P->bptr[i];
    for (int c = 0; c < 3; ++c) {
      int64_t r = 3 * i + c;
      int64_t start = 9 * P->bptr[i] + 3 * len * c;
      row_ptr[r] = start;
      for (int64_t k = 0; k < len; ++k)
        for (int d = 0; d < 3; ++d) col[start + 3 * k + d] = (int32_t)(3 * P->bcol[P->bptr[i] + k] + d);
    }
  }
  row_ptr[3 * P->nbasis] = 9 * P->bptr[P->nbasis];
}

/* Position of basis j in the row of basis i (binary search). */
static int64_t find_in_row(const pattern* P, int64_t i, int64_t j) {
  int64_t lo = P->bptr[i], hi = P->bptr[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (P->bcol[mid] == j) return mid - P->bptr[i];
    if (P->bcol[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static void add_block(const pattern* P, int64_t i, int64_t j, const double* blk, double* val) {
  int64_t k = find_in_row(P, i, j);
  int64_t len = P->bptr[i + 1] - P->bptr[i];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) val[9 * P->bptr[i] + 3 * len * c + 3 * k + d] += blk[c * 3 + d];
}

int ora_pattern(const ora_problem* pr, int64_t* row_ptr, int32_t* col) {
  if (check_problem(pr) < 0) return -1;
  pattern P;
  if (pattern_build(pr, &P) < 0) return -1;
  pattern_to_csr(&P, row_ptr, col);
  pattern_free(&P);
  return 0;
}

int ora_assemble(const ora_problem* pr, int64_t* row_ptr, int32_t* col, double* val) {
  if (check_problem(pr) < 0) return -1;
  pattern P;
  if (pattern_build(pr, &P) < 0) return -1;
  pattern_to_csr(&P, row_ptr, col);
  memset(val, 0, sizeof(double) * 9 * P.bptr[P.nbasis]);
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nlt = pr->t.degree + 1;
  int nls = nlx * nly, nl = nls * nlt;
  int nx = P.su.n;
  int64_t ns = (int64_t)P.su.n * P.sv.n;
  double* Ke = malloc(sizeof(double) * (size_t)nl * nl * 9);
  if (!Ke) { pattern_free(&P); return -1; }
  for (int et = 0; et < P.st.nel; ++et)
    for (int ey = 0; ey < P.sv.nel; ++ey)
      for (int ex = 0; ex < P.su.nel; ++ex) {
        if (ora_element_stiffness(pr, ex, ey, et, Ke) < 0) { free(Ke); pattern_free(&P); return -1; }
        for (int a = 0; a < nl; ++a)
          for (int b = 0; b < nl; ++b) {
            int lta = a / nls, lsa = a % nls, ltb = b / nls, lsb = b % nls;
            int64_t i = (int64_t)(P.st.first[et] + lta) * ns + (int64_t)(P.sv.first[ey] + lsa / nlx) * nx +
                        (P.su.first[ex] + lsa % nlx);
            int64_t j = (int64_t)(P.st.first[et] + ltb) * ns + (int64_t)(P.sv.first[ey] + lsb / nlx) * nx +
                        (P.su.first[ex] + lsb % nlx);
            add_block(&P, i, j, Ke + ((size_t)a * nl + b) * 9, val);
          }
      }
  free(Ke);
  pattern_free(&P);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Element-list assembly for the timed CPU baseline: the element stiffness   */
/* of each listed 3D element added into val on a CSR pattern given by the    */
/* caller (the oracle's own ora_pattern), entry positions found by binary     */
/* search in the rows. No second formula: the same element integrals as      */
/* ora_assemble, restricted to a list, so that a caller can run lists of one */
/* element colour (elements that share no basis function) on several threads.*/
/* ------------------------------------------------------------------------ */
static int64_t csr_find(const int64_t* row_ptr, const int32_t* col, int64_t r, int64_t c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < c) lo = mid + 1; else hi = mid;
  }
  return (lo < row_ptr[r + 1] && col[lo] == c) ? lo : -1;
}

int ora_assemble_elements(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const int32_t* elems,
                          int32_t n, double* val) {
  if (check_problem(pr) < 0) return -1;
  support1d su, sv, st;
  if (support_build(&pr->u, &su) < 0 || support_build(&pr->v, &sv) < 0 || support_build(&pr->t, &st) < 0) return -1;
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nlt = pr->t.degree + 1;
  int nls = nlx * nly, nl = nls * nlt;
  int nx = su.n;
  int64_t ns = (int64_t)su.n * sv.n;
  double* Ke = malloc(sizeof(double) * (size_t)nl * nl * 9);
  int rc = Ke ? 0 : -1;
  for (int32_t k = 0; k < n && rc == 0; ++k) {
    int ex = elems[3 * k], ey = elems[3 * k + 1], et = elems[3 * k + 2];
    if (ora_element_stiffness(pr, ex, ey, et, Ke) < 0) { rc = -1; break; }
    for (int a = 0; a < nl && rc == 0; ++a)
      for (int b = 0; b < nl; ++b) {
        int lta = a / nls, lsa = a % nls, ltb = b / nls, lsb = b % nls;
        int64_t i = (int64_t)(st.first[et] + lta) * ns + (int64_t)(sv.first[ey] + lsa / nlx) * nx +
                    (su.first[ex] + lsa % nlx);
        int64_t j = (int64_t)(st.first[et] + ltb) * ns + (int64_t)(sv.first[ey] + lsb / nlx) * nx +
                    (su.first[ex] + lsb % nlx);
        for (int c = 0; c < 3; ++c) {
          int64_t q = csr_find(row_ptr, col, 3 * i + c, 3 * j);
          if (q < 0) { rc = -1; break; }
          for (int d = 0; d < 3; ++d) val[q + d] += Ke[((size_t)a * nl + b) * 9 + c * 3 + d];
        }
        if (rc) break;
      }
  }
  free(Ke);
  support_free(&su);
  support_free(&sv);
  support_free(&st);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Every block of the rows of one in-plane function: K^{(it, is), (jt, js)}  */
/* for all thickness functions it, jt and every in-plane js in the box       */
/* |jx - ix| <= p_u, |jy - iy| <= p_v, by the integrand of ora_element_       */
/* stiffness restricted to the row functions (it, is): the 3D elements in     */
/* the support of is, every ply piece, the tensor Gauss rule. Layout:         */
/* out[(((it * nt + jt) * nby + (jy - by0)) * nbx + (jx - bx0)) * 9 + c*3+d], */
/* box[0..3] = bx0, nbx, by0, nby.                                            */
/* ------------------------------------------------------------------------ */
int ora_inplane_row_blocks(const ora_problem* pr, int64_t is, int32_t* box, double* out) {
  if (check_problem(pr) < 0) return -1;
  support1d su, sv, st;
  if (support_build(&pr->u, &su) < 0 || support_build(&pr->v, &sv) < 0 || support_build(&pr->t, &st) < 0) return -1;
  int rc = 0;
  const int nx = su.n, ny = sv.n, nt = st.n;
  const int ix = (int)(is % nx), iy = (int)(is / nx);
  const int pu = pr->u.degree, pv = pr->v.degree;
  const int bx0 = ix - pu > 0 ? ix - pu : 0, bx1 = ix + pu + 1 < nx ? ix + pu + 1 : nx;
  const int by0 = iy - pv > 0 ? iy - pv : 0, by1 = iy + pv + 1 < ny ? iy + pv + 1 : ny;
  const int nbx = bx1 - bx0, nby = by1 - by0;
  box[0] = bx0; box[1] = nbx; box[2] = by0; box[3] = nby;
  memset(out, 0, sizeof(double) * 9 * (size_t)nt * nt * nbx * nby);
  const int nlx = pu + 1, nly = pv + 1, nlt = pr->t.degree + 1, nls = nlx * nly;
  int nqu = nq_or_default(pr->nq_u, pu), nqv = nq_or_default(pr->nq_v, pv), nqt = nq_or_default(pr->nq_t, pr->t.degree);
  double xu[64], wu[64], xv[64], wv[64], xt[64], wt[64];
  ora_gauss(nqu, xu, wu);
  ora_gauss(nqv, xv, wv);
  ora_gauss(nqt, xt, wt);
  double (*B)[6][3] = malloc(sizeof(double) * 18 * nls * nlt);
  if (!B) rc = -1;
  inplane_point ip;
  for (int ey = sv.elo[iy]; ey <= sv.ehi[iy] && rc == 0; ++ey)
    for (int ex = su.elo[ix]; ex <= su.ehi[ix] && rc == 0; ++ex) {
      double ua, ub, va, vb;
      int f;
      element_of(&pr->u, ex, &ua, &ub, &f);
      element_of(&pr->v, ey, &va, &vb, &f);
      for (int et = 0; et < st.nel && rc == 0; ++et) {
        double z0[512], z1[512];
        int ply[512];
        int npieces = ply_pieces(pr, et, z0, z1, ply, 512);
        if (npieces < 0) { rc = -1; break; }
        for (int pc = 0; pc < npieces && rc == 0; ++pc) {
          int l = ply[pc];
          double D[36];
          ora_rotated_D(pr->C21 + 21 * pr->ply_material[l], pr->ply_angle[l], D);
          for (int a = 0; a < nqu && rc == 0; ++a)
            for (int b = 0; b < nqv && rc == 0; ++b) {
              double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[a]);
              double eta = va + 0.5 * (vb - va) * (1.0 + xv[b]);
              if (eval_inplane(pr, ex, ey, xi, eta, &ip) < 0) { rc = -1; break; }
              const int li = (iy - ip.fy) * nlx + (ix - ip.fx);
              for (int g = 0; g < nqt; ++g) {
                double z = z0[pc] + 0.5 * (z1[pc] - z0[pc]) * (1.0 + xt[g]);
                double T[8], dT[8];
                int ft;
                if (ora_basis1d_eval(&pr->t, et, z, T, dT, &ft) < 0) { rc = -1; break; }
                const double wq = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * wt[g] * 0.5 * (z1[pc] - z0[pc]);
                const double w = wq * ip.detJ;
                for (int lt = 0; lt < nlt; ++lt)
                  for (int ls = 0; ls < nls; ++ls) {
                    double grad[3];
                    grad3(&ip, ls, T[lt], dT[lt], grad);
                    strain_matrix(grad, B[lt * nls + ls]);
                  }
                for (int lt = 0; lt < nlt; ++lt)
                  for (int ltj = 0; ltj < nlt; ++ltj)
                    for (int lsj = 0; lsj < nls; ++lsj) {
                      const int jx = ip.fx + lsj % nlx, jy = ip.fy + lsj / nlx;
                      const size_t o = (((size_t)(ft + lt) * nt + (ft + ltj)) * nby + (jy - by0)) * nbx + (jx - bx0);
                      add_btdb(w, B[lt * nls + li], D, B[ltj * nls + lsj], out + o * 9);
                    }
              }
            }
        }
      }
    }
  free(B);
  support_free(&su);
  support_free(&sv);
  support_free(&st);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* One block K^{ij}: the same integrand, summed over the 3D elements (and   */
/* their ply pieces) in the intersection of the two supports.               */
/* ------------------------------------------------------------------------ */
int ora_block(const ora_problem* pr, int64_t i, int64_t j, double* out9) {
  if (check_problem(pr) < 0) return -1;
  support1d su, sv, st;
  if (support_build(&pr->u, &su) < 0 || support_build(&pr->v, &sv) < 0 || support_build(&pr->t, &st) < 0) return -1;
  int nx = su.n;
  int64_t ns = (int64_t)su.n * sv.n;
  int64_t nb = ns * st.n;
  memset(out9, 0, sizeof(double) * 9);
  if (i < 0 || j < 0 || i >= nb || j >= nb) { support_free(&su); support_free(&sv); support_free(&st); return -1; }
  int it = (int)(i / ns), iy = (int)((i % ns) / nx), ix = (int)((i % ns) % nx);
  int jt = (int)(j / ns), jy = (int)((j % ns) / nx), jx = (int)((j % ns) % nx);
  int nqu = nq_or_default(pr->nq_u, pr->u.degree), nqv = nq_or_default(pr->nq_v, pr->v.degree);
  int nqt = nq_or_default(pr->nq_t, pr->t.degree);
  double xu[64], wu[64], xv[64], wv[64], xt[64], wt[64];
  ora_gauss(nqu, xu, wu);
  ora_gauss(nqv, xv, wv);
  ora_gauss(nqt, xt, wt);
  int nlx = pr->u.degree + 1;
  inplane_point ip;
  for (int et = st.elo[it]; et <= st.ehi[it]; ++et) {
    if (et < st.elo[jt] || et > st.ehi[jt]) continue;
    double z0[512], z1[512];
    int ply[512];
    int npieces = ply_pieces(pr, et, z0, z1, ply, 512);
    for (int ey = sv.elo[iy]; ey <= sv.ehi[iy]; ++ey) {
      if (ey < sv.elo[jy] || ey > sv.ehi[jy]) continue;
      for (int ex = su.elo[ix]; ex <= su.ehi[ix]; ++ex) {
        if (ex < su.elo[jx] || ex > su.ehi[jx]) continue;
        double ua, ub, va, vb;
        int f;
        element_of(&pr->u, ex, &ua, &ub, &f);
        element_of(&pr->v, ey, &va, &vb, &f);
        for (int pc = 0; pc < npieces; ++pc) {
          double D[36];
          int l = ply[pc];
          ora_rotated_D(pr->C21 + 21 * pr->ply_material[l], pr->ply_angle[l], D);
          for (int a = 0; a < nqu; ++a)
            for (int b = 0; b < nqv; ++b) {
              double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[a]);
              double eta = va + 0.5 * (vb - va) * (1.0 + xv[b]);
              eval_inplane(pr, ex, ey, xi, eta, &ip);
              int li = (iy - ip.fy) * nlx + (ix - ip.fx), lj = (jy - ip.fy) * nlx + (jx - ip.fx);
              for (int g = 0; g < nqt; ++g) {
                double z = z0[pc] + 0.5 * (z1[pc] - z0[pc]) * (1.0 + xt[g]);
                double T[8], dT[8];
                int ft;
                ora_basis1d_eval(&pr->t, et, z, T, dT, &ft);
                double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * wt[g] * 0.5 * (z1[pc] - z0[pc]) * ip.detJ;
                double gi[3], gj[3];
                grad3(&ip, li, T[it - ft], dT[it - ft], gi);
                grad3(&ip, lj, T[jt - ft], dT[jt - ft], gj);
                double Bi[6][3], Bj[6][3];
                strain_matrix(gi, Bi);
                strain_matrix(gj, Bj);
                add_btdb(w, Bi, D, Bj, out9);
              }
            }
        }
      }
    }
  }
  support_free(&su);
  support_free(&sv);
  support_free(&st);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Split form, Section 3: Eq. B_2 splits B^i = B_1^{i_s} T^{i_t} +          */
/* B_2^{i_s} T'^{i_t}; Eq. P integrates the in-plane part per layer, Eq. Q  */
/* the thickness part per layer, and Eq. Km_2 sums their products. Dense    */
/* per-layer P and Q: small problems only.                                  */
/* ------------------------------------------------------------------------ */
int ora_assemble_split(const ora_problem* pr, int64_t* row_ptr, int32_t* col, double* val) {
  if (check_problem(pr) < 0) return -1;
  pattern P;
  if (pattern_build(pr, &P) < 0) return -1;
  int nx = P.su.n, ny = P.sv.n, nt = P.st.n;
  int64_t ns = (int64_t)nx * ny;
  if (ns > 3000 || nt > 600) { pattern_free(&P); return -1; }
  pattern_to_csr(&P, row_ptr, col);
  memset(val, 0, sizeof(double) * 9 * P.bptr[P.nbasis]);
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nls = nlx * nly, nlt = pr->t.degree + 1;
  int nqu = nq_or_default(pr->nq_u, pr->u.degree), nqv = nq_or_default(pr->nq_v, pr->v.degree);
  int nqt = nq_or_default(pr->nq_t, pr->t.degree);
  double xu[64], wu[64], xv[64], wv[64], xt[64], wt[64];
  ora_gauss(nqu, xu, wu);
  ora_gauss(nqv, xv, wv);
  ora_gauss(nqt, xt, wt);
  /* Pl[((is*ns + js)*4 + ab)*9 + c*3 + d], ab = 0:11, 1:12, 2:21, 3:22 */
  double* Pl = malloc(sizeof(double) * (size_t)ns * ns * 36);
  double* Ql = malloc(sizeof(double) * (size_t)nt * nt * 4);
  if (!Pl || !Ql) { free(Pl); free(Ql); pattern_free(&P); return -1; }
  inplane_point ip;
  for (int l = 0; l < pr->n_plies; ++l) {
    double D[36];
    ora_rotated_D(pr->C21 + 21 * pr->ply_material[l], pr->ply_angle[l], D);
    /* Eq. P for this layer */
    memset(Pl, 0, sizeof(double) * (size_t)ns * ns * 36);
    for (int ey = 0; ey < P.sv.nel; ++ey)
      for (int ex = 0; ex < P.su.nel; ++ex) {
        double ua, ub, va, vb;
        int f;
        element_of(&pr->u, ex, &ua, &ub, &f);
        element_of(&pr->v, ey, &va, &vb, &f);
        for (int a = 0; a < nqu; ++a)
          for (int b = 0; b < nqv; ++b) {
            double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[a]);
            double eta = va + 0.5 * (vb - va) * (1.0 + xv[b]);
            eval_inplane(pr, ex, ey, xi, eta, &ip);
            double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * ip.detJ;
            for (int li = 0; li < nls; ++li)
              for (int lj = 0; lj < nls; ++lj) {
                int64_t is = (int64_t)(ip.fy + li / nlx) * nx + ip.fx + li % nlx;
                int64_t js = (int64_t)(ip.fy + lj / nlx) * nx + ip.fx + lj % nlx;
                double B1i[6][3], B2i[6][3], B1j[6][3], B2j[6][3];
                double v1i[3], v2i[3], v1j[3], v2j[3];
                grad3(&ip, li, 1.0, 0.0, v1i);
                grad3(&ip, li, 0.0, 1.0, v2i);
                grad3(&ip, lj, 1.0, 0.0, v1j);
                grad3(&ip, lj, 0.0, 1.0, v2j);
                strain_matrix(v1i, B1i);
                strain_matrix(v2i, B2i);
                strain_matrix(v1j, B1j);
                strain_matrix(v2j, B2j);
                double* dst = Pl + ((size_t)is * ns + js) * 36;
                add_btdb(w, B1i, D, B1j, dst + 0);
                add_btdb(w, B1i, D, B2j, dst + 9);
                add_btdb(w, B2i, D, B1j, dst + 18);
                add_btdb(w, B2i, D, B2j, dst + 27);
              }
          }
      }
    /* Eq. Q for this layer: integrate over the pieces of every thickness
     * element that belong to layer l. */
    memset(Ql, 0, sizeof(double) * (size_t)nt * nt * 4);
    for (int et = 0; et < P.st.nel; ++et) {
      double z0[512], z1[512];
      int ply[512];
      int npieces = ply_pieces(pr, et, z0, z1, ply, 512);
      for (int pc = 0; pc < npieces; ++pc) {
        if (ply[pc] != l) continue;
        for (int g = 0; g < nqt; ++g) {
          double z = z0[pc] + 0.5 * (z1[pc] - z0[pc]) * (1.0 + xt[g]);
          double T[8], dT[8];
          int ft;
          ora_basis1d_eval(&pr->t, et, z, T, dT, &ft);
          double w = wt[g] * 0.5 * (z1[pc] - z0[pc]);
          for (int a = 0; a < nlt; ++a)
            for (int b = 0; b < nlt; ++b) {
              double* q = Ql + ((size_t)(ft + a) * nt + (ft + b)) * 4;
              q[0] += w * T[a] * T[b];
              q[1] += w * T[a] * dT[b];
              q[2] += w * dT[a] * T[b];
              q[3] += w * dT[a] * dT[b];
            }
        }
      }
    }
    /* Eq. Km_2 for this layer, over every block of the pattern */
    for (int64_t i = 0; i < P.nbasis; ++i) {
      int64_t it = i / ns, is = i % ns;
      int64_t len = P.bptr[i + 1] - P.bptr[i];
      for (int64_t k = 0; k < len; ++k) {
        int64_t j = P.bcol[P.bptr[i] + k];
        int64_t jt = j / ns, js = j % ns;
        const double* pp = Pl + ((size_t)is * ns + js) * 36;
        const double* qq = Ql + ((size_t)it * nt + jt) * 4;
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int ab = 0; ab < 4; ++ab) s += pp[ab * 9 + c * 3 + d] * qq[ab];
            val[9 * P.bptr[i] + 3 * len * c + 3 * k + d] += s;
          }
      }
    }
  }
  free(Pl);
  free(Ql);
  pattern_free(&P);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient of L = sum_{stored (r, s)} gbar_rs K_rs with respect to the     */
/* Voigt matrix D_l of every ply (all 36 entries taken as independent).     */
/* K is linear in D_l (Eq. Km_0), so                                        */
/*   dL/dD_l[I][J] = sum_{elements, points in ply l} w |DF|                  */
/*                   sum_{i,j,c,d} gbar_{3i+c, 3j+d} B^i[I][c] B^j[J][d].    */
/* out: n_plies x 36, row-major [l][I*6+J].                                  */
/* ------------------------------------------------------------------------ */
int ora_adjoint_D(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const double* gbar,
                  double* out) {
  if (check_problem(pr) < 0) return -1;
  pattern P;
  if (pattern_build(pr, &P) < 0) return -1;
  int nlx = pr->u.degree + 1, nly = pr->v.degree + 1, nlt = pr->t.degree + 1;
  int nls = nlx * nly, nl = nls * nlt;
  int nx = P.su.n;
  int64_t ns = (int64_t)P.su.n * P.sv.n;
  int nqu = nq_or_default(pr->nq_u, pr->u.degree), nqv = nq_or_default(pr->nq_v, pr->v.degree);
  int nqt = nq_or_default(pr->nq_t, pr->t.degree);
  double xu[64], wu[64], xv[64], wv[64], xt[64], wt[64];
  ora_gauss(nqu, xu, wu);
  ora_gauss(nqv, xv, wv);
  ora_gauss(nqt, xt, wt);
  memset(out, 0, sizeof(double) * 36 * pr->n_plies);
  double* gl = malloc(sizeof(double) * (size_t)nl * nl * 9);   /* local cotangent blocks */
  double (*B)[6][3] = malloc(sizeof(double) * 18 * nl);
  int64_t* gidx = malloc(sizeof(int64_t) * nl);
  if (!gl || !B || !gidx) { free(gl); free(B); free(gidx); pattern_free(&P); return -1; }
  inplane_point ip;
  for (int et = 0; et < P.st.nel; ++et)
    for (int ey = 0; ey < P.sv.nel; ++ey)
      for (int ex = 0; ex < P.su.nel; ++ex) {
        double ua, ub, va, vb, ta, tb;
        int fx, fy, ft;
        element_of(&pr->u, ex, &ua, &ub, &fx);
        element_of(&pr->v, ey, &va, &vb, &fy);
        element_of(&pr->t, et, &ta, &tb, &ft);
        for (int a = 0; a < nl; ++a) {
          int lt = a / nls, ls = a % nls;
          gidx[a] = (int64_t)(ft + lt) * ns + (int64_t)(fy + ls / nlx) * nx + (fx + ls % nlx);
        }
        /* the cotangent restricted to this element's function pairs, read from the CSR */
        for (int a = 0; a < nl; ++a)
          for (int b = 0; b < nl; ++b) {
            int64_t k = find_in_row(&P, gidx[a], gidx[b]);
            int64_t len = P.bptr[gidx[a] + 1] - P.bptr[gidx[a]];
            for (int c = 0; c < 3; ++c) {
              int64_t r = 3 * gidx[a] + c;
              for (int d = 0; d < 3; ++d) gl[((size_t)a * nl + b) * 9 + c * 3 + d] = gbar[row_ptr[r] + 3 * k + d];
              (void)len;
            }
          }
        double z0[512], z1[512];
        int ply[512];
        int npieces = ply_pieces(pr, et, z0, z1, ply, 512);
        for (int pc = 0; pc < npieces; ++pc) {
          double* o = out + 36 * ply[pc];
          for (int qa = 0; qa < nqu; ++qa)
            for (int qb = 0; qb < nqv; ++qb) {
              double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[qa]);
              double eta = va + 0.5 * (vb - va) * (1.0 + xv[qb]);
              eval_inplane(pr, ex, ey, xi, eta, &ip);
              for (int g = 0; g < nqt; ++g) {
                double z = z0[pc] + 0.5 * (z1[pc] - z0[pc]) * (1.0 + xt[g]);
                double T[8], dT[8];
                int f2;
                ora_basis1d_eval(&pr->t, et, z, T, dT, &f2);
                double w = wu[qa] * 0.5 * (ub - ua) * wv[qb] * 0.5 * (vb - va) * wt[g] * 0.5 * (z1[pc] - z0[pc]) * ip.detJ;
                for (int lt = 0; lt < nlt; ++lt)
                  for (int ls = 0; ls < nls; ++ls) {
                    double grad[3];
                    grad3(&ip, ls, T[lt], dT[lt], grad);
                    strain_matrix(grad, B[lt * nls + ls]);
                  }
                for (int a = 0; a < nl; ++a)
                  for (int b = 0; b < nl; ++b) {
                    const double* gb = gl + ((size_t)a * nl + b) * 9;
                    for (int c = 0; c < 3; ++c)
                      for (int d = 0; d < 3; ++d) {
                        double gv = gb[c * 3 + d];
                        if (gv == 0.0) continue;
                        for (int I = 0; I < 6; ++I) {
                          double bi = B[a][I][c];
                          if (bi == 0.0) continue;
                          for (int J = 0; J < 6; ++J) o[I * 6 + J] += w * gv * bi * B[b][J][d];
                        }
                      }
                  }
              }
            }
        }
      }
  free(gl);
  free(B);
  free(gidx);
  pattern_free(&P);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* d/dtheta of the rotated Voigt matrix: the product rule applied to the    */
/* four rotation factors of C'_ijkl = R_ip R_jq R_kr R_ls C_pqrs.          */
/* ------------------------------------------------------------------------ */
void ora_rotated_D_dtheta(const double* C21, double theta, double* D36) {
  double Dm[6][6];
  int k = 0;
  for (int I = 0; I < 6; ++I)
    for (int J = I; J < 6; ++J) {
      Dm[I][J] = C21[k];
      Dm[J][I] = C21[k];
      ++k;
    }
  double c = cos(theta), s = sin(theta);
  double R[3][3] = {{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}};
  double dR[3][3] = {{-s, -c, 0.0}, {c, -s, 0.0}, {0.0, 0.0, 0.0}};
  static const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      int i = pairs[I][0], j = pairs[I][1], kk = pairs[J][0], l = pairs[J][1];
      double sum = 0.0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
          for (int r = 0; r < 3; ++r)
            for (int t = 0; t < 3; ++t) {
              double f = dR[i][p] * R[j][q] * R[kk][r] * R[l][t] + R[i][p] * dR[j][q] * R[kk][r] * R[l][t] +
                         R[i][p] * R[j][q] * dR[kk][r] * R[l][t] + R[i][p] * R[j][q] * R[kk][r] * dR[l][t];
              sum += f * Dm[voigt(p, q)][voigt(r, t)];
            }
      D36[I * 6 + J] = sum;
    }
}

/* ------------------------------------------------------------------------ */
/* Gradients of L = sum gbar_rs K_rs with respect to the material constants */
/* (21 per material, the upper triangle of C in the material frame) and to  */
/* every ply angle. K is linear in each D_l, and D_l = rot(C_m, theta_l) is  */
/* linear in C_m, so                                                        */
/*   dL/dC_m[k]   = sum_{plies l of m} < dL/dD_l, rot(e_k, theta_l) >        */
/*   dL/dtheta_l  = < dL/dD_l, d rot(C_m, theta)/dtheta at theta_l >         */
/* with <A, B> = sum_IJ A_IJ B_IJ and e_k the k-th unit constant vector.     */
/* dD may be NULL.                                                          */
/* ------------------------------------------------------------------------ */
int ora_adjoint(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const double* gbar, double* dD,
                double* dC, double* dtheta) {
  double* g = malloc(sizeof(double) * 36 * (pr->n_plies > 0 ? pr->n_plies : 1));
  if (!g) return -1;
  if (ora_adjoint_D(pr, row_ptr, col, gbar, g) < 0) { free(g); return -1; }
  memset(dC, 0, sizeof(double) * 21 * pr->n_materials);
  for (int l = 0; l < pr->n_plies; ++l) {
    const int m = pr->ply_material[l];
    double R[36], e[21];
    for (int k = 0; k < 21; ++k) {
      memset(e, 0, sizeof e);
      e[k] = 1.0;
      ora_rotated_D(e, pr->ply_angle[l], R);
      double acc = 0.0;
      for (int t = 0; t < 36; ++t) acc += g[36 * l + t] * R[t];
      dC[21 * m + k] += acc;
    }
    ora_rotated_D_dtheta(pr->C21 + 21 * m, pr->ply_angle[l], R);
    double acc = 0.0;
    for (int t = 0; t < 36; ++t) acc += g[36 * l + t] * R[t];
    dtheta[l] = acc;
  }
  if (dD) memcpy(dD, g, sizeof(double) * 36 * pr->n_plies);
  free(g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The in-plane operators of Eq. P for one in-plane pair (i_s, j_s) and the  */
/* material of ply l: P_ab = int B_a^{i_s T} D_l B_b^{j_s} |DF| over the     */
/* shared in-plane elements, with B_1 the strain matrix of (S_x, S_y, 0) and */
/* B_2 that of (0, 0, S) (Eq. B_2). out: 4 x 3 x 3, blocks 11, 12, 21, 22.   */
/* ------------------------------------------------------------------------ */
int ora_inplane_P(const ora_problem* pr, int l, int64_t is, int64_t js, double* out36) {
  if (check_problem(pr) < 0 || l < 0 || l >= pr->n_plies) return -1;
  support1d su, sv;
  if (support_build(&pr->u, &su) < 0 || support_build(&pr->v, &sv) < 0) return -1;
  int nx = su.n;
  int64_t ns = (int64_t)su.n * sv.n;
  memset(out36, 0, sizeof(double) * 36);
  if (is < 0 || js < 0 || is >= ns || js >= ns) { support_free(&su); support_free(&sv); return -1; }
  int iy = (int)(is / nx), ix = (int)(is % nx), jy = (int)(js / nx), jx = (int)(js % nx);
  int nqu = nq_or_default(pr->nq_u, pr->u.degree), nqv = nq_or_default(pr->nq_v, pr->v.degree);
  double xu[64], wu[64], xv[64], wv[64];
  ora_gauss(nqu, xu, wu);
  ora_gauss(nqv, xv, wv);
  int nlx = pr->u.degree + 1;
  double D[36];
  ora_rotated_D(pr->C21 + 21 * pr->ply_material[l], pr->ply_angle[l], D);
  inplane_point ip;
  for (int ey = sv.elo[iy]; ey <= sv.ehi[iy]; ++ey) {
    if (ey < sv.elo[jy] || ey > sv.ehi[jy]) continue;
    for (int ex = su.elo[ix]; ex <= su.ehi[ix]; ++ex) {
      if (ex < su.elo[jx] || ex > su.ehi[jx]) continue;
      double ua, ub, va, vb;
      int f;
      element_of(&pr->u, ex, &ua, &ub, &f);
      element_of(&pr->v, ey, &va, &vb, &f);
      for (int a = 0; a < nqu; ++a)
        for (int b = 0; b < nqv; ++b) {
          double xi = ua + 0.5 * (ub - ua) * (1.0 + xu[a]);
          double eta = va + 0.5 * (vb - va) * (1.0 + xv[b]);
          if (eval_inplane(pr, ex, ey, xi, eta, &ip) < 0) { support_free(&su); support_free(&sv); return -1; }
          int li = (iy - ip.fy) * nlx + (ix - ip.fx), lj = (jy - ip.fy) * nlx + (jx - ip.fx);
          double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * ip.detJ;
          double gi1[3], gi2[3], gj1[3], gj2[3];
          grad3(&ip, li, 1.0, 0.0, gi1);
          grad3(&ip, li, 0.0, 1.0, gi2);
          grad3(&ip, lj, 1.0, 0.0, gj1);
          grad3(&ip, lj, 0.0, 1.0, gj2);
          double Bi1[6][3], Bi2[6][3], Bj1[6][3], Bj2[6][3];
          strain_matrix(gi1, Bi1);
          strain_matrix(gi2, Bi2);
          strain_matrix(gj1, Bj1);
          strain_matrix(gj2, Bj2);
          add_btdb(w, Bi1, D, Bj1, out36);
          add_btdb(w, Bi1, D, Bj2, out36 + 9);
          add_btdb(w, Bi2, D, Bj1, out36 + 18);
          add_btdb(w, Bi2, D, Bj2, out36 + 27);
        }
    }
  }
  support_free(&su);
  support_free(&sv);
  return 0;
}
