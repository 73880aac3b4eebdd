/*
 * CPU oracle for the stiffness matrix of an extruded layered solid.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library. The product
 * (paper_1905_05417_gb300 and its CUDA library) never includes, links or calls
 * anything here, and nothing here includes the product's headers.
 *
 * What it computes (Antolin, "Fast assembly of Galerkin matrices for 3D solid
 * laminated composites", Sections 2.1-2.4 and 3):
 *   K^{ij} = sum_l int_{Omega_l} B^{iT} D_l B^j |DF| dxi            (Eq. Km_0)
 * element by element with tensor Gauss rules (Section 2.4), and, as a second
 * formula for small cases, the split form
 *   K^{ij} = sum_l sum_{ab} P_{l,ab}^{i_s j_s} Q_{l,ab}^{i_t j_t}   (Eq. Km_2)
 * with P from Eq. P and Q from Eq. Q.
 *
 * Conventions (the same ones the library documents, restated here):
 *   - in-plane basis S^{i_s}, i_s = iy*nx + ix; thickness basis T^{i_t};
 *     3D basis index i = i_t*n_s + i_s (Assumption 1); DOF = 3*i + c.
 *   - the map is the extrusion F(xi) = S(xi^1, xi^2) + xi^3 a (Eq. extrusion):
 *     S planar (x, y, 0) or a surface in R^3, a = e_z unless given; the
 *     thickness coordinate xi^3 runs over the thickness knots (physical z
 *     when a = e_z).
 *   - ply 0 starts at the first thickness knot; plies are stacked upwards.
 *   - materials: 21 Voigt constants (upper triangle, row-major, order
 *     11,22,33,12,13,23, engineering shear) in the material frame; a ply with
 *     angle theta has its fibre axis 1 at +theta about +z from global x.
 */
#ifndef LAM_ORACLE_H
#define LAM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BSPLINE = 0, ORA_LAGRANGE = 1 };

typedef struct {
  int32_t kind;          /* ORA_BSPLINE or ORA_LAGRANGE */
  int32_t degree;
  int32_t n_knots;       /* B-spline: knot-vector length; Lagrange: number of breakpoints */
  const double* knots;   /* B-spline: open knot vector; Lagrange: element breakpoints */
} ora_basis1d;

typedef struct {
  ora_basis1d u, v;        /* in-plane directions xi^1 (x-index) and xi^2 (y-index) */
  const double* ctrl;      /* n_s x ctrl_dim control points, i_s = iy*nx + ix */
  const double* weights;   /* n_s NURBS weights or NULL */
  ora_basis1d t;           /* thickness basis in physical z */
  int32_t n_plies;
  const double* ply_thickness;
  const int32_t* ply_material;
  const double* ply_angle;  /* radians */
  int32_t n_materials;
  const double* C21;        /* n_materials x 21 */
  int32_t nq_u, nq_v, nq_t; /* Gauss points per element direction (<= 0: degree + 1) */
  int32_t ctrl_dim;         /* 2: planar mid-surface, ctrl n_s x 2; 3: surface S in R^3, ctrl n_s x 3
                               (Eq. extrusion); 0 reads as 2 */
  const double* extrusion;  /* the constant extrusion direction a of Eq. extrusion (3 values), NULL = e_z */
} ora_problem;

/* Gauss-Legendre rule with n points on [-1, 1], ascending abscissae. */
int ora_gauss(int32_t n, double* x, double* w);

/* Number of functions / elements of a 1D basis. */
int32_t ora_nfun(const ora_basis1d* b);
int32_t ora_nel(const ora_basis1d* b);

/* Values and first derivatives of the degree+1 functions of element e at x
 * (x inside the element); *first receives the index of the first function. */
int ora_basis1d_eval(const ora_basis1d* b, int32_t e, double x, double* val, double* der, int32_t* first);

/* D of a ply: the 6x6 Voigt matrix of C rotated by theta about z. */
void ora_rotated_D(const double* C21, double theta, double* D36);

/* Sizes of the 3D problem. */
int ora_sizes(const ora_problem* pr, int64_t* n_dof, int64_t* nnz);

/* Sparsity pattern only (the oracle's own construction by element supports). */
int ora_pattern(const ora_problem* pr, int64_t* row_ptr, int32_t* col);

/* Full standard assembly (Eq. Km_0, Section 2.4) into the oracle's own CSR. */
int ora_assemble(const ora_problem* pr, int64_t* row_ptr, int32_t* col, double* val);

/* Full split assembly (Eq. Km_2 with Eq. P and Eq. Q, one P per ply). */
int ora_assemble_split(const ora_problem* pr, int64_t* row_ptr, int32_t* col, double* val);

/* The element stiffness of each listed 3D element (elems: n triples ex, ey,
 * et) added into val on the CSR pattern row_ptr / col (from ora_pattern): the
 * integrals of ora_assemble restricted to a list, for the timed CPU baseline.
 * Calls may run concurrently on lists of elements that share no basis
 * function (one element colour). */
int ora_assemble_elements(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const int32_t* elems,
                          int32_t n, double* val);

/* Every 3x3 block of the rows of in-plane function is (all thickness
 * functions it, jt; in-plane js in the box |jx - ix| <= p_u, |jy - iy| <= p_v,
 * clipped): out[(((it * n_t + jt) * nby + (jy - by0)) * nbx + (jx - bx0)) * 9
 * + c * 3 + d] with box = {bx0, nbx, by0, nby}; out holds
 * 9 n_t^2 (2 p_u + 1)(2 p_v + 1) doubles at most. The same integrand as
 * ora_element_stiffness, restricted to the row functions (it, is). */
int ora_inplane_row_blocks(const ora_problem* pr, int64_t is, int32_t* box, double* out);

/* One 3x3 block K^{ij} (row-major, [c][d]) for 3D basis indices i, j. */
int ora_block(const ora_problem* pr, int64_t i, int64_t j, double* out9);

/* Element stiffness of 3D element (ex, ey, et), all ply pieces inside it:
 * out is nl x nl blocks of 3x3, nl = (pu+1)(pv+1)(q+1), local order
 * (lt, ly, lx) with lx fastest. Returns nl, or -1 on error. */
int ora_element_stiffness(const ora_problem* pr, int32_t ex, int32_t ey, int32_t et, double* out);

/* Gradient of L = sum gbar_rs K_rs (gbar on the oracle's CSR pattern) with
 * respect to every ply's Voigt matrix D_l, all 36 entries independent:
 * out[l * 36 + I * 6 + J]. */
int ora_adjoint_D(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const double* gbar,
                  double* out);

/* d/dtheta of ora_rotated_D (product rule over the four rotation factors). */
void ora_rotated_D_dtheta(const double* C21, double theta, double* D36);

/* dL/dC (n_materials x 21), dL/dtheta (n_plies) and optionally dL/dD
 * (n_plies x 36, may be NULL) for L = sum gbar * K on the oracle's pattern. */
int ora_adjoint(const ora_problem* pr, const int64_t* row_ptr, const int32_t* col, const double* gbar, double* dD,
                double* dC, double* dtheta);

/* Eq. P for the in-plane pair (is, js) and ply l's material: 4 blocks of 3x3
 * (11, 12, 21, 22), row-major. */
int ora_inplane_P(const ora_problem* pr, int l, int64_t is, int64_t js, double* out36);

#ifdef __cplusplus
}
#endif
#endif
