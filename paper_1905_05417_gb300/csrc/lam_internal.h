// Internal plan representation shared by the host plan builder (lam_plan.cpp)
// and the CUDA side (lam_kernels.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lam.h"

namespace lam {

constexpr int kMaxDegree = 7;

// One 1D basis with its element structure (Section 2.2).
struct Basis {
  int kind = LAM_BSPLINE;
  int p = 1;
  std::vector<double> knots;
  int n = 0;                     // functions
  int nel = 0;                   // elements (nonempty knot spans / breakpoint intervals)
  std::vector<double> ea, eb;    // element bounds
  std::vector<int> span;         // B-spline knot-span index of each element
  std::vector<int> first;        // first function of each element
  std::vector<int> elo, ehi;     // elements in the support of each function
  std::vector<int> lo, len;      // neighbour range [lo, lo + len) of each function
  int colors = 1;                // elements >= colors apart share no function
};

// A (thickness element, ply) piece: Eq. C_layers restricted to one element.
struct Piece {
  int elem;
  int ply;
  int cfg;
  double z0, z1;
};

struct Device;  // device mirror, defined in lam_kernels.cu

struct Plan {
  Basis u, v, t;
  std::vector<double> ctrl;      // n_s x 2 (x, y)
  std::vector<double> weights;   // n_s, empty when polynomial
  // general extrusion F = S + xi^3 a (Eq. extrusion): S in R^3 and/or a != e_z
  bool shell = false;
  std::vector<double> ctrl3;     // n_s x 3 (x, y, z), shells only
  double extrusion[3] = {0.0, 0.0, 1.0};
  std::vector<lam_ply> plies;
  std::vector<lam_material> mats;
  int nqu = 0, nqv = 0, nqt = 0;
  double class_tol = 1e-13;
  int arith = LAM_ARITH_FP64;    // lam_options.arith

  // Gauss-Legendre rules on [-1, 1]
  std::vector<double> gxu, gwu, gxv, gwv, gxt, gwt;
  // in-plane 1D tables: [e][q][k][2] (value, d/dxi) and weights [e][q] (Gauss weight x half length)
  std::vector<double> tabU, tabV, wU, wV;

  // (material, angle) configurations: Section 3, one P set per distinct D
  std::vector<int> ply_cfg;
  std::vector<int> cfg_mat;
  std::vector<double> cfg_angle;
  std::vector<double> cfgD;      // [m][6][6]
  std::vector<double> cfgE;      // [m][c*3+d][a*3+b] = D_m[V(c,a)][V(d,b)]
  std::vector<double> cfgCb;     // [m][i][j][p][r] = C{e_i, e_j}_{pr} = C_{pirj} (rotated 4th-order tensor)
  bool monoclinic = true;

  // thickness pieces and their 1D tables
  std::vector<Piece> pieces;
  std::vector<int> piece_begin;  // per thickness element, size t.nel + 1
  std::vector<double> tabT;      // [piece][q][k][2] (T, dT/dz)
  std::vector<double> wT;        // [piece][q]

  // in-plane pattern: row i_s has len_s(i_s) = len_x * len_y neighbours
  int64_t ns = 0, nnz_s = 0;
  std::vector<int64_t> LSb;      // prefix of len_s, size ns + 1
  // thickness pattern
  int64_t nt = 0, nnz_t = 0;
  std::vector<int64_t> LTb;      // prefix of len_t, size nt + 1
  std::vector<int> tp_row, tp_col;       // thickness pair -> (i_t, j_t)
  std::vector<int> tp_e0, tp_e1;         // shared thickness elements of the pair
  std::vector<int64_t> tp_A;             // 9 * LTb[i_t] * nnz_s: CSR start of thickness row i_t's slab
  std::vector<int> tp_lt, tp_k;          // len_t(i_t) and k_t of the pair

  // combine classes: thickness pairs with equal Q vectors
  int ncls = 0;
  std::vector<int> cls_rep;              // representative pair of each class
  std::vector<int> pair_cls;             // class of every thickness pair
  std::vector<std::vector<int>> cls_cfgs;  // configurations with nonzero Q of every class
  // streaming combine, in thickness chunks: chunk ch covers thickness rows
  // [ck_it[ch], ck_it[ch + 1]); the classes of its pairs take slots
  // 0 .. ck_nslot[ch] - 1 of the row's shared-memory slices; its terms
  // (slot, configuration, representative pair), sorted by configuration, are
  // ck_term[ch] .. ck_term[ch + 1] - 1; ckt_first marks the first term of a slot.
  int kc_slots = 0;                      // slots that fit in shared memory
  std::vector<int> ck_it, ck_term, ck_nslot;
  std::vector<int> ckt_slot, ckt_cfg, ckt_rep, ckt_first;
  std::vector<int> pair_slot;            // slot of every thickness pair within its chunk
  // ... and for monoclinic plates, per chunk, the terms of the slots that are
  // computed for each entry kind (block: Q_11, Q_22; off: Q_12, Q_21): terms
  // ck_sterm[ch] .. + ck_nblk[ch] - 1 for the block kind, then the off kind's up
  // to ck_sterm[ch + 1] - 1 (sorted by configuration, cks_first marking the
  // first term of a slot); slots that share a kind's Q terms with an earlier slot
  // are copied from it: ck_copy[ch] .. ck_copy[ch + 1] - 1, ckc_dst = 2 slot +
  // kind, ckc_src = the source slot
  std::vector<int> ck_sterm, ck_nblk, cks_slot, cks_cfg, cks_rep, cks_first;
  std::vector<int> ck_copy, ckc_dst, ckc_src;
  double q_scale[4] = {0.0, 0.0, 0.0, 0.0};  // largest |Q_ab| over every pair and configuration
  std::vector<int> cls_term_begin;       // size ncls + 1
  std::vector<int> cls_terms;            // configuration ids with nonzero Q
  std::vector<int> cls_occ_begin;        // size ncls + 1
  std::vector<int64_t> occ_A;            // 9 * LTb[i_t] * nnz_s of each occurrence
  std::vector<int> occ_lt, occ_k, occ_it;  // len_t(i_t), k_t, i_t of each occurrence
  std::vector<double> host_q;            // host Q per pair [pair][cfg][4] (classification only)

  // adjoint (lam_adjoint): for every ply, the thickness pairs whose common
  // support meets the ply, with Eq. Q restricted to that ply, divided by the
  // power of two adj_qscale[type] (types: T T, T T', T' T, T' T')
  std::vector<int> adj_begin;            // size n_plies + 1
  std::vector<int> adj_pair;             // thickness pair of each term
  std::vector<double> adj_q;             // [term][4]
  std::vector<float> adj_qdf;            // [term][8]: float pairs (hi[4], lo[4]) of adj_q
  double adj_qscale[4] = {1.0, 1.0, 1.0, 1.0};
  int adj_max_terms = 0;
  // chain rule through Eq. D: D_l = M(theta_l) C_m M(theta_l)^T
  std::vector<double> ply_M, ply_dM;     // [l][36]: Bond matrix and its derivative in theta
  std::vector<double> mat_C;             // [m][36]: material matrix
  std::vector<int> ply_mat;              // material of each ply

  // colourings
  std::vector<int> col2_begin, col2_elem;  // in-plane elements (ey * nel_u + ex)
  std::vector<int> col3_begin, col3_elem;  // 3D elements ((et * nel_v + ey) * nel_u + ex)

  int64_t n_dof = 0, nnz = 0;

  Device* dev = nullptr;
  int device_id = -1;
  bool cfg_dirty = true;         // configuration tables must be (re)uploaded
  int cfg_version = 0;           // incremented by lam_plan_update (batches check it)
  int chunk_ctas = 0;            // CTAs per SM the thickness chunks are sized for (0: by registers)

  // profiler (lam_profile_*): events are cudaEvent_t, kept opaque here
  struct Pending {
    int kind;
    int count;
    void* start;
    void* stop;
  };
  bool prof_enabled = false;
  int64_t prof_launches[LAM_KERNEL_KINDS] = {};
  double prof_ms[LAM_KERNEL_KINDS] = {};
  int64_t prof_h2d = 0, prof_d2h = 0;
  std::vector<Pending> prof_pending;
  std::vector<void*> prof_free_events;
};

// Launch geometry of the combine shared by host and device code: the
// streaming form keeps a row's class slices in shared memory (one 512-thread
// CTA per row, two per SM), a chunk of thickness rows at a time; rows of more
// than 512 / 9 in-plane neighbours take the class-major form.
inline int max_len_s(const Plan& P) {
  int mx = 0, my = 0;
  for (int v : P.u.len) mx = mx > v ? mx : v;
  for (int v : P.v.len) my = my > v ? my : v;
  return mx * my;
}
// threads of a streaming-combine CTA (one per (c, k_s, d) of the largest row)
inline int kcs_block(const Plan& P) {
  const int t = ((9 * max_len_s(P) + 31) / 32) * 32;
  return t < 128 ? 128 : t;
}
// CTAs of that size an SM holds at 64 registers per thread, and the shared
// memory each of them may use (228 KB per SM, 1 KB reserved per CTA)
inline int kcs_ctas_per_sm(const Plan& P) {
  int n = 65536 / (64 * kcs_block(P));
  if (n > 2048 / kcs_block(P)) n = 2048 / kcs_block(P);
  return n < 1 ? 1 : (n > 8 ? 8 : n);
}
// shared memory a thickness chunk may use: the SM's share of the CTAs it is sized for
inline size_t kcs_budget(const Plan& P) {
  const int n = P.chunk_ctas > 0 ? P.chunk_ctas : kcs_ctas_per_sm(P);
  return (size_t)(233472 / n) - 1024;
}
inline int kcs_stride(const Plan& P) { return 9 * max_len_s(P); }
inline int kcs_max_terms(const Plan& P) {
  int mt = 1;
  for (size_t ch = 0; ch + 1 < P.ck_term.size(); ++ch) mt = mt > P.ck_term[ch + 1] - P.ck_term[ch] ? mt : P.ck_term[ch + 1] - P.ck_term[ch];
  for (size_t ch = 0; ch + 1 < P.ck_sterm.size(); ++ch)
    mt = mt > P.ck_sterm[ch + 1] - P.ck_sterm[ch] ? mt : P.ck_sterm[ch + 1] - P.ck_sterm[ch];
  return mt;
}
// largest copy list of a chunk (entries of slots taken from a source slot)
inline int kcs_max_copies(const Plan& P) {
  int mc = 1;
  for (size_t ch = 0; ch + 1 < P.ck_copy.size(); ++ch) mc = mc > P.ck_copy[ch + 1] - P.ck_copy[ch] ? mc : P.ck_copy[ch + 1] - P.ck_copy[ch];
  return mc;
}
inline size_t kcs_smem(const Plan& P) {
  int slots = 1;
  for (int v : P.ck_nslot) slots = slots > v ? slots : v;
  // slices, then per term of a chunk: Q (4 float pairs or 4 doubles), slot, first flag, configuration
  return (size_t)slots * kcs_stride(P) * sizeof(double) + (size_t)kcs_max_terms(P) * (32 + 12) +
         (size_t)kcs_max_copies(P) * 8 + 16;
}
inline bool use_stream(const Plan& P) { return 9 * max_len_s(P) <= 512 && !P.ck_nslot.empty(); }

// lam_plan.cpp
lam_status build_plan(Plan& P, const lam_inplane* inplane, const lam_basis1d* thickness, const lam_ply* plies,
                      int32_t n_plies, const lam_material* materials, int32_t n_materials, const lam_options* opt);
lam_status rebuild_configs(Plan& P);
void build_chunks(Plan& P);
void set_error(const char* fmt, ...);
void free_device(Plan& P);  // lam_kernels.cu

}  // namespace lam

struct lam_plan {
  lam::Plan p;
};
