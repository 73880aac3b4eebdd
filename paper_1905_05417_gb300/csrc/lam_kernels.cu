// CUDA (sm_103a) kernels and the device-side C ABI of the stiffness assembly.
//
// Split path (Section 3 of Antolin 2019, Eq. Km_2):
//   K-b  kb_thickness  Q_{m,ab}^{i_t j_t} = sum_{plies l of configuration m}
//                      int_{ply l} tau_a^{i_t} tau_b^{j_t} dz   (Eq. Q; tau_1 = T, tau_2 = T')
//   K-a  ka_local64    configuration-free in-plane Gram blocks per element
//                      G_{ab}^{i_s j_s} = int g_a^{i_s} g_b^{j_s} |DF| dxi,
//                      g = (dS/dx, dS/dy, S)   (pull-back of Eq. gradient), FP64
//                      (ka_local: double-float; ka_inplane: accumulated per pair,
//                      for the allocation-free entry point); kg_rows sums them
//                      per in-plane pair
//   K-c  kc_ws         P_{m,ab}[c][d] = sum D_m[V(c,a)][V(d,b)] G_{ab} (Eq. P with a
//                      homogeneous ply), then K = sum_m sum_ab P_{m,ab} Q_{m,ab}
//                      written straight into the CSR values, FP64, warp-specialised
//                      (kc_stream: the double-float pass and the fallback;
//                      kc_combine: the class-major form for rows of many neighbours)
// General extrusions (Eq. extrusion): ka_shell64 / ka_shell (6 x 6 Gram blocks),
// kp_shell64 / kp_shell (P per configuration), the combine reading P.
// Standard path (Section 2.4): K-d kd_standard, one CTA per 3D element.
// Adjoint: adj_* (dL/dD_l, dL/dC, dL/dtheta). Batches: kb_batch, ka_batch, kc_batch.
// Pattern: kp_row_ptr / kp_col_ind.
#include <cuda_runtime.h>
#include <mutex>
#include <string>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lam_internal.h"

namespace lam {

#define LAM_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t err__ = (call);                                                                \
    if (err__ != cudaSuccess) {                                                                \
      ::lam::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(err__), __FILE__, __LINE__); \
      return LAM_ERR_CUDA;                                                                     \
    }                                                                                          \
  } while (0)

struct Device {
  // in-plane
  double *tabU = nullptr, *tabV = nullptr, *wU = nullptr, *wV = nullptr;
  int *firstU = nullptr, *firstV = nullptr;
  int *loX = nullptr, *lenX = nullptr, *loY = nullptr, *lenY = nullptr;
  double *ctrl = nullptr, *weights = nullptr;
  int64_t* LSb = nullptr;
  int* col2_elem = nullptr;
  // thickness
  int *loT = nullptr, *lenT = nullptr, *firstT = nullptr;
  int64_t* LTb = nullptr;
  double *tabT = nullptr, *wT = nullptr;
  int *piece_begin = nullptr, *piece_cfg = nullptr;
  int *tp_row = nullptr, *tp_col = nullptr, *tp_e0 = nullptr, *tp_e1 = nullptr;
  int64_t* tp_A = nullptr;
  int *tp_lt = nullptr, *tp_k = nullptr;
  // classes
  int *cls_term_begin = nullptr, *cls_terms = nullptr, *cls_occ_begin = nullptr, *term_rep = nullptr;
  int64_t* occ_A = nullptr;
  int *occ_lt = nullptr, *occ_k = nullptr, *occ_it = nullptr;
  // configurations
  double* cfgE = nullptr;
  // standard path
  int* col3_elem = nullptr;
  // workspace
  int *eloX = nullptr, *ehiX = nullptr, *eloY = nullptr, *ehiY = nullptr;
  int* pair_cls = nullptr;
  int *ck_it = nullptr, *ck_term = nullptr, *ck_nslot = nullptr, *pair_slot = nullptr;
  int *ckt_slot = nullptr, *ckt_cfg = nullptr, *ckt_rep = nullptr, *ckt_first = nullptr;
  int *ck_sterm = nullptr, *ck_nblk = nullptr, *cks_slot = nullptr, *cks_cfg = nullptr, *cks_rep = nullptr,
      *cks_first = nullptr, *ck_copy = nullptr, *ckc_dst = nullptr, *ckc_src = nullptr;
  float2* qdf = nullptr;  // float pairs of q

  double* EG = nullptr;  // element Gram blocks: n_el x pairs x 9
  double* Grow = nullptr;  // assembled Gram blocks of every in-plane pair: nnz_s x 9 (FP64 combine)
  // per in-plane pair, the element blocks its G sums (kg_rows): gsum_off[gsum_begin[pr] ..
  // gsum_begin[pr + 1]) = 2 x (EG position of the block) + 1 if read transposed; null if not built
  int* gsum_begin = nullptr;
  int* gsum_off = nullptr;
  int* kc_flag = nullptr;      // streaming combine: FP64 re-pass flag, then the largest exponent
  float2* cfgEdf = nullptr;    // float pairs of cfgE
  double* cfgCb = nullptr;     // Appendix A bracket tensors per configuration
  double* bfree_EP = nullptr;  // element operators of the Voigt-free construction (lazily allocated)
  // general extrusion (Eq. extrusion): surface control points, element Gram
  // blocks of the six gradient parts, P of every configuration (lazily allocated)
  double* ctrl3 = nullptr;
  double* shellEG = nullptr;   // n_el x 36 x pairs
  double* shellP = nullptr;    // n_cfg x nnz_s x 36
  size_t shellP_elems = 0;
  unsigned long long* shell_pmax = nullptr;  // 4 block maxima of |P|
  // adjoint of a general extrusion: the assembled 6 x 6 Gram blocks, and unit scales
  double* adj_G36 = nullptr;   // nnz_s x 36
  float2* adj_G36df = nullptr;  // its scaled float pairs
  double* adj_gscale36 = nullptr;  // the 9 scales of adj_G36df
  // K-b runs on a stream of its own beside K-a, forked from and joined to the caller's stream
  cudaStream_t kb_stream = nullptr;
  cudaEvent_t kb_fork = nullptr, kb_join = nullptr;
  float2* shell_Edf = nullptr;  // cfgE 2^-kE per configuration, float pairs (configuration tables)
  int* shell_kE = nullptr;
  int n_sm = 0;
  int smem_optin = 0;    // largest dynamic shared memory of one CTA
  double* q = nullptr;   // nnz_t x n_cfg x 4
  bool q_valid = false;  // q holds Eq. Q of the current configurations (recomputed after lam_plan_update)
  // adjoint: geometry tables and workspace (allocated by the first lam_adjoint)
  bool adj_ready = false;
  bool adj_g_cached = false;       // adj_G / adj_Gdf / scales hold this plan's scaled Gram blocks
  double* adj_W = nullptr;         // low rank: n_t x n_s x 27 (G v per thickness function)
  double* adj_X = nullptr;         // low rank: nnz_t x 81 (u^T G v per thickness pair)
  int *adj_begin = nullptr, *adj_pair = nullptr;
  double* adj_q = nullptr;
  float* adj_qdf = nullptr;
  double* adj_G = nullptr;         // assembled G / gscale, nnz_s x 9
  float2* adj_Gdf = nullptr;       // float pairs of adj_G
  unsigned long long* adj_gmax = nullptr;  // 9 maxima of |G_ab| (bit patterns), then 9 scales (doubles)
  double* adj_partial = nullptr;   // n_plies x n_chunks x 81
  double* adj_plyC = nullptr;      // n_plies x 21
  int* adj_flag = nullptr;         // set when the double-float pass produced a non-finite partial
  // adjoint: chain-rule tables (configuration dependent)
  double *ply_M = nullptr, *ply_dM = nullptr, *mat_C = nullptr;
  int* ply_mat = nullptr;
  // host-output staging
  double* stage[2] = {nullptr, nullptr};
  size_t stage_elems = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_done[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  std::vector<void*> allocs;      // geometry tables and in-plane workspace (plan lifetime)
  std::vector<void*> cfg_allocs;  // configuration tables (replaced after lam_plan_update)
};

// Every device allocation of the library goes through here. Fault injection
// for tests of the error paths (host side only, no device fault): with
// LAM_FAIL_ALLOC=n in the environment, the n-th allocation counted from the
// moment the variable took its current value fails as an out-of-memory
// cudaMalloc would, and the caller's usual clean-up runs.
static cudaError_t device_alloc(void** p, size_t bytes) {
  static std::mutex mu;
  static std::string armed;
  static long count = 0;
  const char* env = getenv("LAM_FAIL_ALLOC");
  {
    std::lock_guard<std::mutex> lock(mu);
    const std::string v = env ? env : "";
    if (v != armed) {
      armed = v;
      count = 0;
    }
    if (!v.empty()) {
      const long n = atol(v.c_str());
      if (n > 0 && ++count == n) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
    }
  }
  return cudaMalloc(p, bytes);
}

template <typename T>
static lam_status upload(Plan& P, std::vector<void*>& list, T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
  void* p = nullptr;
  cudaError_t e = device_alloc(&p, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LAM_ERR_OOM : LAM_ERR_CUDA;
  }
  list.push_back(p);
  if (!src.empty()) {
    LAM_CUDA(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    P.prof_h2d += (int64_t)(src.size() * sizeof(T));
  }
  *dst = static_cast<T*>(p);
  return LAM_OK;
}

static lam_status alloc_dev(std::vector<void*>& list, double** dst, size_t n) {
  void* p = nullptr;
  cudaError_t e = device_alloc(&p, std::max<size_t>(n, 1) * sizeof(double));
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu doubles) failed: %s", n, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LAM_ERR_OOM : LAM_ERR_CUDA;
  }
  list.push_back(p);
  *dst = static_cast<double*>(p);
  return LAM_OK;
}

// ---------------------------------------------------------------------------
// Profiler: an event pair on the launching stream around each launch group.
// ---------------------------------------------------------------------------
static cudaEvent_t prof_event(Plan& P) {
  if (!P.prof_free_events.empty()) {
    cudaEvent_t e = static_cast<cudaEvent_t>(P.prof_free_events.back());
    P.prof_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

static cudaEvent_t prof_begin(Plan& P, cudaStream_t s) {
  if (!P.prof_enabled) return nullptr;
  cudaEvent_t a = prof_event(P);
  if (a) cudaEventRecord(a, s);
  return a;
}

static void prof_end(Plan& P, int kind, int count, cudaStream_t s, cudaEvent_t a) {
  P.prof_launches[kind] += count;
  if (!P.prof_enabled || !a) return;
  cudaEvent_t b = prof_event(P);
  if (!b) return;
  cudaEventRecord(b, s);
  P.prof_pending.push_back(Plan::Pending{kind, count, a, b});
}

static void prof_collect(Plan& P) {
  for (auto& pd : P.prof_pending) {
    cudaEvent_t a = static_cast<cudaEvent_t>(pd.start), b = static_cast<cudaEvent_t>(pd.stop);
    float ms = 0.0f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
      P.prof_ms[pd.kind] += ms;
    P.prof_free_events.push_back(a);
    P.prof_free_events.push_back(b);
  }
  P.prof_pending.clear();
}

static void free_cfg_tables(Device& D) {
  for (void* p : D.cfg_allocs) cudaFree(p);
  D.cfg_allocs.clear();
}

void free_device(Plan& P) {
  if (!P.dev) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (P.device_id >= 0) cudaSetDevice(P.device_id);
  cudaDeviceSynchronize();
  prof_collect(P);
  for (void* e : P.prof_free_events) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  P.prof_free_events.clear();
  free_cfg_tables(*P.dev);
  for (void* p : P.dev->allocs) cudaFree(p);
  for (int k = 0; k < 2; ++k) {
    if (P.dev->stage[k]) cudaFree(P.dev->stage[k]);
    if (P.dev->ev_done[k]) cudaEventDestroy(P.dev->ev_done[k]);
    if (P.dev->ev_copied[k]) cudaEventDestroy(P.dev->ev_copied[k]);
  }
  if (P.dev->copy_stream) cudaStreamDestroy(P.dev->copy_stream);
  if (P.dev->kb_stream) cudaStreamDestroy(P.dev->kb_stream);
  if (P.dev->kb_fork) cudaEventDestroy(P.dev->kb_fork);
  if (P.dev->kb_join) cudaEventDestroy(P.dev->kb_join);
  if (P.dev->shellP) cudaFree(P.dev->shellP);
  delete P.dev;
  P.dev = nullptr;
  if (cur >= 0) cudaSetDevice(cur);
}

// ---------------------------------------------------------------------------
// Launch geometry
// ---------------------------------------------------------------------------

static int kc_block(const Plan& P) { return ((9 * max_len_s(P) + 31) / 32) * 32; }

static int kc_np(const Plan& P) { return (P.monoclinic && !P.shell) ? 2 : 4; }

static int kc_gs_cap(const Plan& P) { return (9 * max_len_s(P) + 1) & ~1; }

static size_t kc_smem(const Plan& P) {
  const int ncfg = (int)P.cfg_mat.size();
  size_t b = 0;
  b += (size_t)kc_gs_cap(P) * sizeof(double);                     // G row
  b += (size_t)ncfg * kc_np(P) * kc_block(P) * sizeof(double);    // per-thread P
  b += (size_t)P.cls_terms.size() * 4 * sizeof(double);           // Q of every class term
  b += (size_t)P.nnz_t * 3 * sizeof(int64_t);                     // CSR bases per (c, occurrence)
  b += (size_t)(2 * (P.ncls + 1) + P.cls_terms.size()) * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

static int ka_nls(const Plan& P) { return (P.u.p + 1) * (P.v.p + 1); }
static int ka_npl(const Plan& P) { return ka_nls(P) * (ka_nls(P) + 1) / 2; }
static int ka_block(const Plan& P) {
  int np = ka_nls(P) * (ka_nls(P) + 1) / 2;
  return np >= 256 ? 256 : ((np + 31) / 32) * 32;
}
static size_t ka_smem(const Plan& P) {
  const int nqs = P.nqu * P.nqv, nls = ka_nls(P);
  size_t b = (size_t)nqs * nls * 6 * sizeof(double) + (size_t)nqs * 8 * sizeof(double);
  b += (size_t)(nls * (nls + 1) / 2) * 2;
  return (b + 15) & ~(size_t)15;
}
// K-d: point values of the in-plane element, and the element's weighted
// thickness values (most pieces of a thickness element x points x functions x 2)
static size_t kd_tw(const Plan& P) {
  int mp = 1;
  for (size_t e = 0; e + 1 < P.piece_begin.size(); ++e) mp = std::max(mp, P.piece_begin[e + 1] - P.piece_begin[e]);
  return (size_t)mp * P.nqt * (P.t.p + 1) * 2 * sizeof(double);
}
static size_t kd_smem(const Plan& P) {
  const int nqs = P.nqu * P.nqv, nls = ka_nls(P);
  if (P.shell) return (size_t)nqs * nls * 4 * sizeof(double) + (size_t)nqs * 16 * sizeof(double) + kd_tw(P);
  return (size_t)nqs * nls * 3 * sizeof(double) + (size_t)nqs * 8 * sizeof(double) + kd_tw(P);
}
// K-a of a general extrusion in FP64: shell_points plus the gradient parts u and w u
static size_t ka_shell64_smem(const Plan& P) {
  const int nqs = P.nqu * P.nqv, nls = ka_nls(P);
  return (size_t)nqs * nls * 16 * sizeof(double) + (size_t)nqs * 16 * sizeof(double);
}
// K-a of a general extrusion: float pairs of u and w u, per point 16 doubles
static size_t ka_shell_smem(const Plan& P) {
  const int nqs = P.nqu * P.nqv, nls = ka_nls(P);
  return (size_t)nqs * nls * 24 * sizeof(float) + (size_t)nqs * 16 * sizeof(double);
}

// ---------------------------------------------------------------------------
// Pattern kernels
// ---------------------------------------------------------------------------
struct PatArgs {
  int64_t ns, nt, n_dof, nnz, nnz_s;
  int nx;
  const int64_t *LSb, *LTb;
  const int *loX, *lenX, *loY, *lenY, *loT, *lenT;
};

// row_ptr(i_t, i_s, c) = 9 LTb[i_t] nnz_s + 9 len_t LSb[i_s] + 3 c len_t len_s
__global__ void kp_row_ptr(PatArgs a, int64_t* __restrict__ row_ptr) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r > a.n_dof) return;
  if (r == a.n_dof) {
    row_ptr[r] = a.nnz;
    return;
  }
  const int64_t i = r / 3, c = r % 3, it = i / a.ns, is = i % a.ns;
  const int64_t lt = a.LTb[it + 1] - a.LTb[it], ls = a.LSb[is + 1] - a.LSb[is];
  row_ptr[r] = 9 * a.LTb[it] * a.nnz_s + 9 * lt * a.LSb[is] + 3 * c * lt * ls;
}

// One block per (i_s, i_t): the 3 rows of that function pair are contiguous.
__global__ void kp_col_ind(PatArgs a, int32_t* __restrict__ col) {
  const int64_t is = blockIdx.x, it = blockIdx.y;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ly = a.lenY[iy], ls = lx * ly;
  const int lt = a.lenT[it];
  const int64_t base = 9 * a.LTb[it] * a.nnz_s + 9 * (int64_t)lt * a.LSb[is];
  const int row_len = 3 * lt * ls, total = 3 * row_len;
  for (int p = threadIdx.x; p < total; p += blockDim.x) {
    const int rem = p % row_len;
    const int kt = rem / (3 * ls), rem2 = rem % (3 * ls);
    const int ks = rem2 / 3, d = rem2 % 3;
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int64_t jt = a.loT[it] + kt;
    col[base + p] = (int32_t)(3 * (jt * a.ns + (int64_t)jy * a.nx + jx) + d);
  }
}

// ---------------------------------------------------------------------------
// K-b: thickness pair integrals (Eq. Q), summed per configuration.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Double-float arithmetic (pairs of floats on the FP32 pipes)
// ---------------------------------------------------------------------------
// a * b added to the double-float accumulator (sh, sl), with a = ah + al and
// b = bh + bl split into float pairs. The product is taken to about 2^-48
// relative (the rounding error of ah * bh by FMA, plus the two cross terms;
// al * bl is below that), the sum by Knuth's two-sum. Intrinsics keep the
// compiler from contracting the error-free transformations.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = t;
}

// g = hi + lo with |g - hi - lo| <= 2^-46 |g| for 2^-80 <= |g| < 2^128: hi is
// g truncated to 24 significant bits, lo the top 23 of the remaining 29 bits,
// both formed from the bits of g with integer and exact float operations (no
// FP64 arithmetic). Smaller magnitudes keep hi only (|g| >= 2^-126) or vanish;
// larger ones, infinities and NaNs give a non-finite hi, which the caller's
// finiteness check turns into the FP64 evaluation. Returns the biased FP64
// exponent of g (0 for zero).
__device__ __forceinline__ int split_df(double g, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(g);
  const unsigned int H = (unsigned int)(b >> 32), Lw = (unsigned int)b;
  const unsigned int sign = H & 0x80000000u;
  const int E = (int)((H >> 20) & 0x7FFu);
  const unsigned int nb = sign | ((unsigned int)(E - 896) << 23) | ((H & 0xFFFFFu) << 3) | (Lw >> 29);
  hi = __int_as_float((int)((E < 897) ? sign : ((E > 1150) ? (sign | 0x7F800000u) : nb)));
  const float r = __fsub_rn(__int_as_float((int)(0x4B000000u | ((Lw & 0x1FFFFFFFu) >> 6))), 8388608.0f);
  const int se = (E >= 943 && E <= 1150) ? (E - 942) : 0;  // exponent field of 2^(E - 1069); 0 gives 0.0f
  lo = __int_as_float(__float_as_int(__fmul_rn(r, __int_as_float(se << 23))) | (int)sign);
  return E;
}

// The split of split_df for the hot loop, in fewer integer operations: valid
// for 2^-80 <= |g| < 2^128 (biased exponent 943 ... 1150); below, hi = lo = 0.
// Above, the result is meaningless: the caller tracks the largest exponent and
// the FP64 pass recomputes everything when it exceeds 1150.
__device__ __forceinline__ int split_df_fast(double g, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(g);
  const unsigned int H = (unsigned int)(b >> 32), Lw = (unsigned int)b;
  const int E = (int)((H >> 20) & 0x7FFu);
  // (H << 3 | Lw >> 29) holds E mod 512 and the top 23 mantissa bits; rebias E by -896
  const unsigned int hb = ((__funnelshift_l(Lw, H, 3) - (384u << 23)) & 0x7FFFFFFFu) | (H & 0x80000000u);
  const unsigned int sb = (hb & 0xFF800000u) - (46u << 23);  // sign * 2^(E - 1069)
  const float r = __fsub_rn(__int_as_float((int)(0x4B000000u | ((Lw >> 6) & 0x7FFFFFu))), 8388608.0f);
  const bool keep = E >= 943;
  hi = keep ? __int_as_float((int)hb) : 0.0f;
  lo = keep ? __fmul_rn(r, __int_as_float((int)sb)) : 0.0f;
  return E;
}

// split_df_fast of g * 2^-k (exact scaling folded into the exponent rebias):
// valid when g * 2^-k lies in [2^-80, 2^128); smaller scaled values give 0.
__device__ __forceinline__ void split_df_off(double g, int k, float& hi, float& lo) {
  const unsigned int H = (unsigned int)__double2hiint(g), Lw = (unsigned int)__double2loint(g);
  const int E = (int)((H >> 20) & 0x7FFu);
  const unsigned int hb =
      ((__funnelshift_l(Lw, H, 3) - (((unsigned int)(384 + k) & 511u) << 23)) & 0x7FFFFFFFu) | (H & 0x80000000u);
  const unsigned int sb = (hb & 0xFF800000u) - (46u << 23);
  const float r = __fsub_rn(__int_as_float((int)(0x4B000000u | ((Lw >> 6) & 0x7FFFFFu))), 8388608.0f);
  const bool keep = E - k >= 943 && E - k <= 1150;
  hi = keep ? __int_as_float((int)hb) : 0.0f;
  lo = keep ? __fmul_rn(r, __int_as_float((int)sb)) : 0.0f;
}

// (p, e) with p + e = a * b to about 2^-47 relative, a and b given as float pairs
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& p, float& e) {
  p = __fmul_rn(ah, bh);
  e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
}

// (sh, sl) += (ph, pl) by Knuth's two-sum on the high parts
__device__ __forceinline__ void df_add(float ph, float pl, float& sh, float& sl) {
  const float t = __fadd_rn(sh, ph);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(ph, z));
  sl = __fadd_rn(sl, __fadd_rn(err, pl));
  sh = t;
}

// The double nearest (to about 2^-47 relative) to the float pair h + l,
// |l| <= ulp(h) / 2, formed from the bits with integer operations and one FMA
// (GB300 converts between float and double at the FP64 rate). |h| is widened
// exactly; l, measured in units of 2^-46 of |h|'s binade, is added to the bit
// pattern (l taken twice as large when h is a power of two and l lowers it into
// the binade below). l is dropped for |h| < 2^-81; h = 0 gives 0.
__device__ __forceinline__ double df_to_double(float h, float l) {
  const unsigned int hb = __float_as_uint(h);
  const unsigned int mag = hb & 0x7FFFFFFFu, sign = hb & 0x80000000u;
  const int eh = (int)(mag >> 23);
  const unsigned long long dh =
      ((unsigned long long)((mag >> 3) + (896u << 20)) << 32) | (unsigned long long)(mag << 29);
  const float lr = __uint_as_float(__float_as_uint(l) ^ sign);  // l relative to the sign of h
  const int se = 300 - eh;                                      // exponent field of 2^(173 - eh)
  const bool use_l = eh >= 46 && se <= 254;
  const float t = __fmaf_rn(lr, __uint_as_float((unsigned int)(use_l ? se : 0) << 23), 12582912.0f);
  long long L = (long long)(int)(__float_as_uint(t) - 0x4B400000u);
  if ((mag & 0x7FFFFFu) == 0u && L < 0) L *= 2;
  const unsigned long long dm = (mag == 0u) ? 0ull : dh + (unsigned long long)(L * 64);
  return __longlong_as_double((long long)(dm | ((unsigned long long)sign << 32)));
}

struct KbArgs {
  int64_t npairs;
  int ncfg, nqt, q1;
  const int *tp_row, *tp_col, *tp_e0, *tp_e1, *firstT, *piece_begin, *piece_cfg;
  const double *tabT, *wT;
  double* q;
  float2* qdf;  // float pairs of q (may be NULL)
};

__device__ __forceinline__ void kb_pair(const KbArgs& a, int64_t pr) {
  double* out = a.q + pr * a.ncfg * 4;
  for (int k = 0; k < a.ncfg * 4; ++k) out[k] = 0.0;
  const int i = a.tp_row[pr], j = a.tp_col[pr];
  for (int e = a.tp_e0[pr]; e <= a.tp_e1[pr]; ++e) {
    const int ia = i - a.firstT[e], jb = j - a.firstT[e];
    for (int pc = a.piece_begin[e]; pc < a.piece_begin[e + 1]; ++pc) {
      double q11 = 0.0, q12 = 0.0, q21 = 0.0, q22 = 0.0;
      for (int g = 0; g < a.nqt; ++g) {
        const double* tb = a.tabT + ((size_t)pc * a.nqt + g) * a.q1 * 2;
        const double w = a.wT[(size_t)pc * a.nqt + g];
        const double Ti = tb[2 * ia], dTi = tb[2 * ia + 1], Tj = tb[2 * jb], dTj = tb[2 * jb + 1];
        // explicit fused multiply-adds: every kernel that inlines this (the plan's
        // K-b, the batch's) rounds alike, whatever the compiler would contract
        const double wTi = w * Ti, wdTi = w * dTi;
        q11 = fma(wTi, Tj, q11);
        q12 = fma(wTi, dTj, q12);
        q21 = fma(wdTi, Tj, q21);
        q22 = fma(wdTi, dTj, q22);
      }
      double* o = out + a.piece_cfg[pc] * 4;
      o[0] += q11;
      o[1] += q12;
      o[2] += q21;
      o[3] += q22;
    }
  }
  if (a.qdf)
    for (int k = 0; k < a.ncfg * 4; ++k) {
      float h, l;
      split_df(out[k], h, l);
      a.qdf[pr * a.ncfg * 4 + k] = make_float2(h, l);
    }
}

__global__ void kb_thickness(KbArgs a) {
  const int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pr < a.npairs) kb_pair(a, pr);
}

// ---------------------------------------------------------------------------
// In-plane point data shared by K-a and K-d: for each Gauss point of the
// in-plane element, the physical gradient (Eq. gradient) and value of every
// local function and the weight w |DF|.
// ---------------------------------------------------------------------------
struct InplaneArgs {
  int nx, nel_u, pu, pv, nqu, nqv;
  const double *tabU, *tabV, *wU, *wV, *ctrl, *weights;
  const int *firstU, *firstV;
  const double* ctrl3;  // general extrusion: n_s x 3 surface control points (else NULL)
  double ax, ay, az;    // the extrusion direction a
};

// pair number of li <= lj, row-major over the upper triangle of n local functions
__device__ __forceinline__ int upper_pair(int a, int b, int n) { return a * n - a * (a - 1) / 2 + (b - a); }

__device__ __forceinline__ void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

// General extrusion F = S(xi1, xi2) + xi3 a (Eq. extrusion; DF independent of
// xi3, Assumption 1): DF = [dS/dxi1 | dS/dxi2 | a]. The rows of DF^-1 are the
// dual vectors g^0 = (A1 x a) / det, g^1 = (a x A0) / det, g^2 = (A0 x A1) / det
// of the columns A0, A1, a, and the gradient of S^k T is T (R_,1 g^0 + R_,2 g^1)
// + T' R g^2 (Eq. gradient pulled back through DF^-T).
//   qs[q * 16 + 0..8]  = g^0, g^1, g^2; [9] = w |DF|; [10..12] = W, W_,1, W_,2
//   ph[(q * nls + k) * 4 + 0..2] = g1 = R_,1 g^0 + R_,2 g^1; [3] = R
constexpr int kShellQ = 16;
__device__ void shell_points(const InplaneArgs& a, int ex, int ey, double* ph, double* qs) {
  const int nlx = a.pu + 1, nly = a.pv + 1, nls = nlx * nly, nqs = a.nqu * a.nqv;
  const int fx = a.firstU[ex], fy = a.firstV[ey];
  for (int t = threadIdx.x; t < nqs; t += blockDim.x) {
    const int qu = t % a.nqu, qv = t / a.nqu;
    const double* tu = a.tabU + ((size_t)ex * a.nqu + qu) * nlx * 2;
    const double* tv = a.tabV + ((size_t)ey * a.nqv + qv) * nly * 2;
    double W = 1.0, W1 = 0.0, W2 = 0.0;
    if (a.weights) {
      W = 0.0;
      for (int ly = 0; ly < nly; ++ly)
        for (int lx = 0; lx < nlx; ++lx) {
          const double w = a.weights[(size_t)(fy + ly) * a.nx + fx + lx];
          const double wu = w * tu[2 * lx], wdu = w * tu[2 * lx + 1];  // explicit FMAs: same rounding in every kernel
          W = fma(wu, tv[2 * ly], W);
          W1 = fma(wdu, tv[2 * ly], W1);
          W2 = fma(wu, tv[2 * ly + 1], W2);
        }
    }
    double A0[3] = {0.0, 0.0, 0.0}, A1[3] = {0.0, 0.0, 0.0};
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        const size_t gi = (size_t)(fy + ly) * a.nx + fx + lx;
        const double N = tu[2 * lx] * tv[2 * ly], N1 = tu[2 * lx + 1] * tv[2 * ly], N2 = tu[2 * lx] * tv[2 * ly + 1];
        double R1 = N1, R2 = N2;
        if (a.weights) {
          const double w = a.weights[gi];
          R1 = w * (N1 * W - N * W1) / (W * W);
          R2 = w * (N2 * W - N * W2) / (W * W);
        }
        const double* X = a.ctrl3 + 3 * gi;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A0[c] += R1 * X[c];
          A1[c] += R2 * X[c];
        }
      }
    const double A2[3] = {a.ax, a.ay, a.az};
    double g0[3], g1[3], g2[3];
    cross3(A1, A2, g0);
    cross3(A2, A0, g1);
    cross3(A0, A1, g2);
    const double det = A0[0] * g0[0] + A0[1] * g0[1] + A0[2] * g0[2], inv = 1.0 / det;
    double* d = qs + (size_t)t * kShellQ;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = g0[c] * inv;
      d[3 + c] = g1[c] * inv;
      d[6 + c] = g2[c] * inv;
    }
    d[9] = a.wU[(size_t)ex * a.nqu + qu] * a.wV[(size_t)ey * a.nqv + qv] * fabs(det);
    d[10] = W;
    d[11] = W1;
    d[12] = W2;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls, k = t % nls;
    const int qu = q % a.nqu, qv = q / a.nqu, lx = k % nlx, ly = k / nlx;
    const double* tu = a.tabU + ((size_t)ex * a.nqu + qu) * nlx * 2;
    const double* tv = a.tabV + ((size_t)ey * a.nqv + qv) * nly * 2;
    const double* d = qs + (size_t)q * kShellQ;
    double R = tu[2 * lx] * tv[2 * ly], R1 = tu[2 * lx + 1] * tv[2 * ly], R2 = tu[2 * lx] * tv[2 * ly + 1];
    if (a.weights) {
      const double w = a.weights[(size_t)(fy + ly) * a.nx + fx + lx], W = d[10];
      const double N = R, N1 = R1, N2 = R2;
      R = w * N / W;
      R1 = w * (N1 * W - N * d[11]) / (W * W);
      R2 = w * (N2 * W - N * d[12]) / (W * W);
    }
    double* f = ph + (size_t)t * 4;
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = d[c] * R1 + d[3 + c] * R2;
    f[3] = R;
  }
  __syncthreads();
}

// qd[q*8 + 0..3] = DF^{-1} (row-major, [k][a]), [4] = w|DF|, [5..7] = W, dW/dxi1, dW/dxi2
__device__ void inplane_points(const InplaneArgs& a, int ex, int ey, double* phi, double* phiw, double* qd) {
  const int nlx = a.pu + 1, nly = a.pv + 1, nls = nlx * nly, nqs = a.nqu * a.nqv;
  const int fx = a.firstU[ex], fy = a.firstV[ey];
  for (int t = threadIdx.x; t < nqs; t += blockDim.x) {
    const int qu = t % a.nqu, qv = t / a.nqu;
    const double* tu = a.tabU + ((size_t)ex * a.nqu + qu) * nlx * 2;
    const double* tv = a.tabV + ((size_t)ey * a.nqv + qv) * nly * 2;
    double W = 1.0, W1 = 0.0, W2 = 0.0;
    if (a.weights) {
      W = 0.0;
      for (int ly = 0; ly < nly; ++ly)
        for (int lx = 0; lx < nlx; ++lx) {
          const double w = a.weights[(size_t)(fy + ly) * a.nx + fx + lx];
          const double wu = w * tu[2 * lx], wdu = w * tu[2 * lx + 1];  // explicit FMAs: same rounding in every kernel
          W = fma(wu, tv[2 * ly], W);
          W1 = fma(wdu, tv[2 * ly], W1);
          W2 = fma(wu, tv[2 * ly + 1], W2);
        }
    }
    double J00 = 0.0, J01 = 0.0, J10 = 0.0, J11 = 0.0;
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        const size_t gi = (size_t)(fy + ly) * a.nx + fx + lx;
        double N = tu[2 * lx] * tv[2 * ly], N1 = tu[2 * lx + 1] * tv[2 * ly], N2 = tu[2 * lx] * tv[2 * ly + 1];
        double R1 = N1, R2 = N2;
        if (a.weights) {
          const double w = a.weights[gi];
          R1 = w * (N1 * W - N * W1) / (W * W);
          R2 = w * (N2 * W - N * W2) / (W * W);
        }
        const double X = a.ctrl[2 * gi], Y = a.ctrl[2 * gi + 1];
        J00 += R1 * X;
        J01 += R2 * X;
        J10 += R1 * Y;
        J11 += R2 * Y;
      }
    const double det = J00 * J11 - J01 * J10;
    const double inv = 1.0 / det;
    double* d = qd + t * 8;
    d[0] = J11 * inv;   // dxi1/dx
    d[1] = -J01 * inv;  // dxi1/dy
    d[2] = -J10 * inv;  // dxi2/dx
    d[3] = J00 * inv;   // dxi2/dy
    d[4] = a.wU[(size_t)ex * a.nqu + qu] * a.wV[(size_t)ey * a.nqv + qv] * fabs(det);
    d[5] = W;
    d[6] = W1;
    d[7] = W2;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls, k = t % nls;
    const int qu = q % a.nqu, qv = q / a.nqu, lx = k % nlx, ly = k / nlx;
    const double* tu = a.tabU + ((size_t)ex * a.nqu + qu) * nlx * 2;
    const double* tv = a.tabV + ((size_t)ey * a.nqv + qv) * nly * 2;
    const double* d = qd + q * 8;
    double R = tu[2 * lx] * tv[2 * ly], R1 = tu[2 * lx + 1] * tv[2 * ly], R2 = tu[2 * lx] * tv[2 * ly + 1];
    if (a.weights) {
      const double w = a.weights[(size_t)(fy + ly) * a.nx + fx + lx], W = d[5];
      const double N = R, N1 = R1, N2 = R2;
      R = w * N / W;
      R1 = w * (N1 * W - N * d[6]) / (W * W);
      R2 = w * (N2 * W - N * d[7]) / (W * W);
    }
    const double gx = d[0] * R1 + d[2] * R2;
    const double gy = d[1] * R1 + d[3] * R2;
    double* f = phi + (size_t)t * 3;
    f[0] = gx;
    f[1] = gy;
    f[2] = R;
    if (phiw) {
      double* fw = phiw + (size_t)t * 3;
      fw[0] = d[4] * gx;
      fw[1] = d[4] * gy;
      fw[2] = d[4] * R;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// K-a: in-plane Gram blocks of one element, accumulated into G (one colour of
// elements per launch, so no two CTAs of a launch touch the same block).
// ---------------------------------------------------------------------------
struct KaArgs {
  InplaneArgs ip;
  const int* elems;
  const int *loX, *lenX, *loY, *lenY;
  const int64_t* LSb;
  double* G;
};

__global__ void __launch_bounds__(256) ka_inplane(KaArgs a) {
  extern __shared__ double sm[];
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  double* phi = sm;
  double* phiw = phi + (size_t)nqs * nls * 3;
  double* qd = phiw + (size_t)nqs * nls * 3;
  const int e = a.elems[blockIdx.x];
  const int ex = e % ip.nel_u, ey = e / ip.nel_u;
  inplane_points(ip, ex, ey, phi, phiw, qd);
  const int npairs = nls * (nls + 1) / 2;
  const int fx = ip.firstU[ex], fy = ip.firstV[ey];
  for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
    // t -> (li <= lj), row-major over the upper triangle
    int li = 0, rem = t;
    while (rem >= nls - li) {
      rem -= nls - li;
      ++li;
    }
    const int lj = li + rem;
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (int q = 0; q < nqs; ++q) {
      const double* A = phiw + ((size_t)q * nls + li) * 3;
      const double* B = phi + ((size_t)q * nls + lj) * 3;
      const double a0 = A[0], a1 = A[1], a2 = A[2], b0 = B[0], b1 = B[1], b2 = B[2];
      acc[0] += a0 * b0;
      acc[1] += a0 * b1;
      acc[2] += a0 * b2;
      acc[3] += a1 * b0;
      acc[4] += a1 * b1;
      acc[5] += a1 * b2;
      acc[6] += a2 * b0;
      acc[7] += a2 * b1;
      acc[8] += a2 * b2;
    }
    const int ix = fx + li % nlx, iy = fy + li / nlx, jx = fx + lj % nlx, jy = fy + lj / nlx;
    const int64_t is = (int64_t)iy * ip.nx + ix, js = (int64_t)jy * ip.nx + jx;
    const int64_t kij = (int64_t)(jy - a.loY[iy]) * a.lenX[ix] + (jx - a.loX[ix]);
    double* g = a.G + (a.LSb[is] + kij) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] += acc[k];
    if (li != lj) {
      const int64_t kji = (int64_t)(iy - a.loY[jy]) * a.lenX[jx] + (ix - a.loX[jx]);
      double* h = a.G + (a.LSb[js] + kji) * 9;
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) h[(ab % 3) * 3 + ab / 3] += acc[ab];
    }
  }
}

// ---------------------------------------------------------------------------
// K-a (single launch): one CTA per in-plane element; the Gram blocks of its
// unordered local pairs (li <= lj) go to EG[(e * npl + pair) * 9 + ab], pair
// numbered row-major over the upper triangle (a pair's 9 entries contiguous,
// so a row's gather reads them in whole sectors). The combine gathers them per row
// in a fixed element order, so the sums are deterministic without colouring.
// ---------------------------------------------------------------------------
struct KaLocalArgs {
  InplaneArgs ip;
  int nel;
  double* EG;
};

// (h, l) = a * b as a normalised float pair (|l| <= ulp(h) / 2).
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float& h, float& l) {
  float p, e;
  df_mul(ah, al, bh, bl, p, e);
  h = __fadd_rn(p, e);
  l = __fsub_rn(e, __fsub_rn(h, p));
}
__device__ __forceinline__ void df_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// The element's point values for the Gram products (Eq. of G_ab: g = (dR/dx,
// dR/dy, R) at every Gauss point), written as float pairs phf / pwf with the
// layout hi0 hi1 hi2 lo0 lo1 lo2 per (point, local function), pwf = w|DF| phf.
//   A  (FP64) per (point, sum): the geometry sums over the element's functions,
//      factorised over the tensor product (sum over x inside, over y outside):
//      the four entries of DF, or for NURBS the nine sums W, dW/dxi_k and the
//      same with w X and w Y, from which DF follows by the quotient rule;
//   P  (FP64) per point: DF^-1 and w|DF| (and 1/W, W_,1/W, W_,2/W);
//   B  (double-float) per (point, function): R, its parametric derivatives,
//      the physical gradient and the weighted copy, on the FP32 pipes.
// DF^-1 is carried as DF^-1 2^-kd and w|DF| as w|DF| 2^-kq (powers of two per
// element, largest entries in [1, 2)), so float pairs hold any geometry scale;
// the Gram block (a, b) is scaled back by 2^(kq + kd ([a < 2] + [b < 2])).
__device__ __forceinline__ void ka_point_values(const InplaneArgs& ip, int ex, int ey, double* phi, double* phiw,
                                                double* qd, int* s_k) {
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  const int fx = ip.firstU[ex], fy = ip.firstV[ey];
  const bool rat = ip.weights != nullptr;
  const int nsum = rat ? 9 : 4;
  double* S = phi;   // phase A results, nqs x nsum (consumed before phase B writes phf)
  double* hc = phiw; // homogeneous control values (w, w X, w Y) of a NURBS element
  if (rat) {
    for (int k = threadIdx.x; k < nls; k += blockDim.x) {
      const size_t gi = (size_t)(fy + k / nlx) * ip.nx + fx + k % nlx;
      const double w = ip.weights[gi];
      hc[k] = w;
      hc[nls + k] = w * ip.ctrl[2 * gi];
      hc[2 * nls + k] = w * ip.ctrl[2 * gi + 1];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nqs * nsum; t += blockDim.x) {
    const int q = t / nsum, sidx = t % nsum;
    const int qu = q % ip.nqu, qv = q / ip.nqu;
    // der: 0 value, 1 d/dxi1, 2 d/dxi2; dat: X, Y (B-spline) or w, w X, w Y (NURBS)
    const int dat = rat ? sidx / 3 : sidx / 2, der = rat ? sidx % 3 : 1 + sidx % 2;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2 + (der == 1 ? 1 : 0);
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2 + (der == 2 ? 1 : 0);
    double acc = 0.0;
    for (int ly = 0; ly < nly; ++ly) {
      double row = 0.0;
      for (int lx = 0; lx < nlx; ++lx) {
        const double c = rat ? hc[dat * nls + ly * nlx + lx]
                             : ip.ctrl[2 * ((size_t)(fy + ly) * ip.nx + fx + lx) + dat];
        row = fma(tu[2 * lx], c, row);
      }
      acc = fma(tv[2 * ly], row, acc);
    }
    S[t] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nqs; q += blockDim.x) {
    const double* sq = S + (size_t)q * nsum;
    double J00, J01, J10, J11, iw = 1.0, r1 = 0.0, r2 = 0.0;
    if (rat) {  // d(A / W) = (dA - (A / W) dW) / W
      iw = 1.0 / sq[0];
      r1 = sq[1] * iw;
      r2 = sq[2] * iw;
      J00 = (sq[4] - sq[3] * r1) * iw;
      J01 = (sq[5] - sq[3] * r2) * iw;
      J10 = (sq[7] - sq[6] * r1) * iw;
      J11 = (sq[8] - sq[6] * r2) * iw;
    } else {
      J00 = sq[0];
      J01 = sq[1];
      J10 = sq[2];
      J11 = sq[3];
    }
    const int qu = q % ip.nqu, qv = q / ip.nqu;
    const double det = J00 * J11 - J01 * J10, inv = 1.0 / det;
    double* d = qd + (size_t)q * 8;
    d[0] = J11 * inv;   // dxi1/dx
    d[1] = -J01 * inv;  // dxi1/dy
    d[2] = -J10 * inv;  // dxi2/dx
    d[3] = J00 * inv;   // dxi2/dy
    d[4] = ip.wU[(size_t)ex * ip.nqu + qu] * ip.wV[(size_t)ey * ip.nqv + qv] * fabs(det);
    d[5] = iw;
    d[6] = r1;
    d[7] = r2;
    int ed = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) ed = max(ed, (__double2hiint(d[k]) >> 20) & 0x7FF);
    atomicMax(&s_k[0], ed);
    atomicMax(&s_k[1], (__double2hiint(d[4]) >> 20) & 0x7FF);
  }
  __syncthreads();
  const int kd = s_k[0] > 0 ? s_k[0] - 1023 : 0, kq = s_k[1] > 0 ? s_k[1] - 1023 : 0;
  float* phf = reinterpret_cast<float*>(phi);
  float* pwf = reinterpret_cast<float*>(phiw);
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls, k = t % nls;
    const int qu = q % ip.nqu, qv = q / ip.nqu, lx = k % nlx, ly = k / nlx;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2 + 2 * lx;
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2 + 2 * ly;
    const double* d = qd + (size_t)q * 8;
    float u0h, u0l, u1h, u1l, v0h, v0l, v1h, v1l;
    split_df_fast(tu[0], u0h, u0l);
    split_df_fast(tu[1], u1h, u1l);
    split_df_fast(tv[0], v0h, v0l);
    split_df_fast(tv[1], v1h, v1l);
    float Rh, Rl, R1h, R1l, R2h, R2l;
    df_prod(u0h, u0l, v0h, v0l, Rh, Rl);
    df_prod(u1h, u1l, v0h, v0l, R1h, R1l);
    df_prod(u0h, u0l, v1h, v1l, R2h, R2l);
    if (rat) {  // R = c N, R_,k = c (N_,k - N W_,k / W), c = w / W
      float ch, cl, rh, rl, th, tl;
      split_df_fast(ip.weights[(size_t)(fy + ly) * ip.nx + fx + lx] * d[5], ch, cl);
      split_df_fast(d[6], rh, rl);
      df_prod(Rh, Rl, -rh, -rl, th, tl);
      df_add(th, tl, R1h, R1l);
      df_norm(R1h, R1l);
      df_prod(R1h, R1l, ch, cl, R1h, R1l);
      split_df_fast(d[7], rh, rl);
      df_prod(Rh, Rl, -rh, -rl, th, tl);
      df_add(th, tl, R2h, R2l);
      df_norm(R2h, R2l);
      df_prod(R2h, R2l, ch, cl, R2h, R2l);
      df_prod(Rh, Rl, ch, cl, Rh, Rl);
    }
    float dh[4], dl[4], wh, wl;
#pragma unroll
    for (int j = 0; j < 4; ++j) split_df_off(d[j], kd, dh[j], dl[j]);
    split_df_off(d[4], kq, wh, wl);
    float gxh, gxl, gyh, gyl;
    df_mul(dh[0], dl[0], R1h, R1l, gxh, gxl);
    df_mac(dh[2], dl[2], R2h, R2l, gxh, gxl);
    df_norm(gxh, gxl);
    df_mul(dh[1], dl[1], R1h, R1l, gyh, gyl);
    df_mac(dh[3], dl[3], R2h, R2l, gyh, gyl);
    df_norm(gyh, gyl);
    float* f = phf + (size_t)t * 6;
    float* fw = pwf + (size_t)t * 6;
    f[0] = gxh;
    f[1] = gyh;
    f[2] = Rh;
    f[3] = gxl;
    f[4] = gyl;
    f[5] = Rl;
    float h, l;
    df_prod(wh, wl, gxh, gxl, h, l);
    fw[0] = h;
    fw[3] = l;
    df_prod(wh, wl, gyh, gyl, h, l);
    fw[1] = h;
    fw[4] = l;
    df_prod(wh, wl, Rh, Rl, h, l);
    fw[2] = h;
    fw[5] = l;
  }
  __syncthreads();
}

__device__ __forceinline__ void ka_elem(const KaLocalArgs& a, int e, double* sm) {
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  double* phi = sm;
  double* phiw = phi + (size_t)nqs * nls * 3;
  double* qd = phiw + (size_t)nqs * nls * 3;
  const int ex = e % ip.nel_u, ey = e / ip.nel_u;
  __shared__ int s_k[2];
  if (threadIdx.x < 2) s_k[threadIdx.x] = 0;
  __syncthreads();
  ka_point_values(ip, ex, ey, phi, phiw, qd, s_k);
  const int kd = s_k[0] > 0 ? s_k[0] - 1023 : 0, kq = s_k[1] > 0 ? s_k[1] - 1023 : 0;
  const float* phf = reinterpret_cast<const float*>(phi);
  const float* pwf = reinterpret_cast<const float*>(phiw);
  const int npl = nls * (nls + 1) / 2;
  double* out = a.EG + (size_t)e * npl * 9;
  for (int t = threadIdx.x; t < npl; t += blockDim.x) {
    int li = 0, rem = t;
    while (rem >= nls - li) {
      rem -= nls - li;
      ++li;
    }
    const int lj = li + rem;
    float sh[9], sl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sh[k] = sl[k] = 0.0f;
    for (int q = 0; q < nqs; ++q) {
      const float* A = pwf + ((size_t)q * nls + li) * 6;
      const float* B = phf + ((size_t)q * nls + lj) * 6;
      float ah[3], al[3], bh[3], bl[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ah[k] = A[k];
        al[k] = A[3 + k];
        bh[k] = B[k];
        bl[k] = B[3 + k];
      }
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) df_mac(ah[x], al[x], bh[y], bl[y], sh[x * 3 + y], sl[x * 3 + y]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float hs = __fadd_rn(sh[k], sl[k]);
      const float ls = __fsub_rn(sl[k], __fsub_rn(hs, sh[k]));
      long long b = __double_as_longlong(df_to_double(hs, ls));
      const int sc = kq + kd * ((k / 3 < 2 ? 1 : 0) + (k % 3 < 2 ? 1 : 0));
      if (b & 0x7FFFFFFFFFFFFFFFll) b += (long long)sc * (1ll << 52);  // times 2^sc, exact
      out[(size_t)t * 9 + k] = __longlong_as_double(b);
    }
  }
}

__global__ void __launch_bounds__(256) ka_local(KaLocalArgs a) {
  extern __shared__ double sm[];
  ka_elem(a, blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// K-a for a general extrusion (Eq. extrusion). B_1 = B(g1) and B_2 = B(R g^2)
// now have three gradient components each (the planar map has (g_x, g_y, 0)
// and (0, 0, R)), so the configuration-free Gram of a local pair has 6 x 6
// entries: G_(alpha a)(beta b) = sum_q w|DF| u^li_(alpha a) u^lj_(beta b),
// u_1 = g1, u_2 = R g^2. EG[(e * npl + pair) * 36 + blk * 9 + a * 3 + b],
// blk = 2 alpha + beta, pair li <= lj; the 36 entries of a pair are
// contiguous, so that the per-row gather reads whole lines. The other order is
// the transposed block: G^ji_(alpha a)(beta b) = G^ij_(beta b)(alpha a). The
// geometry sums and DF^-1 in FP64, the point values and the products in
// double-float, with u_1, u_2 and w|DF| divided by per-element powers of two
// (k1, k2, kq) so that the float pairs keep any geometry scale; block
// (alpha, beta) is scaled back by 2^(kq + k_alpha + k_beta).
// ---------------------------------------------------------------------------
struct KaShellArgs {
  InplaneArgs ip;
  double* EG;
};

__device__ __forceinline__ int exp_field(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// The element's point values of a general extrusion as float pairs
// phf / pwf ([item][12]: hi u_0..u_5, lo u_0..u_5; pwf = w|DF| phf), with
// u = (R_,1 g^0 + R_,2 g^1, R g^2):
//   A (FP64) per (point, sum): dS/dxi1 and dS/dxi2 (three coordinates each),
//     or for NURBS the twelve sums W, dW/dxi_k and the same with w X, w Y, w Z,
//     factorised over the tensor product;
//   P (FP64) per point: the columns of DF, the dual vectors g^k, w|DF|;
//   B (double-float) per (point, function).
// g^0, g^1 enter divided by 2^k1, g^2 by 2^k2 and w|DF| by 2^kq (s_k[0..2]).
__device__ __forceinline__ void ka_shell_point_values(const InplaneArgs& ip, int ex, int ey, float* phf, float* pwf,
                                                      double* qd, int* s_k) {
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  const int fx = ip.firstU[ex], fy = ip.firstV[ey];
  const bool rat = ip.weights != nullptr;
  const int nsum = rat ? 12 : 6;
  double* S = reinterpret_cast<double*>(phf);   // phase A results (consumed before phase B)
  double* hc = reinterpret_cast<double*>(pwf);  // (w, w X, w Y, w Z) of a NURBS element
  if (rat) {
    for (int k = threadIdx.x; k < nls; k += blockDim.x) {
      const size_t gi = (size_t)(fy + k / nlx) * ip.nx + fx + k % nlx;
      const double w = ip.weights[gi];
      hc[k] = w;
#pragma unroll
      for (int c = 0; c < 3; ++c) hc[(1 + c) * nls + k] = w * ip.ctrl3[3 * gi + c];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nqs * nsum; t += blockDim.x) {
    const int q = t / nsum, sidx = t % nsum;
    const int qu = q % ip.nqu, qv = q / ip.nqu;
    // der: 0 value, 1 d/dxi1, 2 d/dxi2; dat: coordinate (B-spline) or w, w X, w Y, w Z (NURBS)
    const int dat = rat ? sidx / 3 : sidx % 3, der = rat ? sidx % 3 : 1 + sidx / 3;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2 + (der == 1 ? 1 : 0);
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2 + (der == 2 ? 1 : 0);
    double acc = 0.0;
    for (int ly = 0; ly < nly; ++ly) {
      double row = 0.0;
      for (int lx = 0; lx < nlx; ++lx) {
        const double c = rat ? hc[dat * nls + ly * nlx + lx]
                             : ip.ctrl3[3 * ((size_t)(fy + ly) * ip.nx + fx + lx) + dat];
        row = fma(tu[2 * lx], c, row);
      }
      acc = fma(tv[2 * ly], row, acc);
    }
    S[t] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nqs; q += blockDim.x) {
    const double* sq = S + (size_t)q * nsum;
    double A0[3], A1[3], iw = 1.0, r1 = 0.0, r2 = 0.0;
    if (rat) {  // d(A / W) = (dA - (A / W) dW) / W
      iw = 1.0 / sq[0];
      r1 = sq[1] * iw;
      r2 = sq[2] * iw;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A0[c] = (sq[3 * (1 + c) + 1] - sq[3 * (1 + c)] * r1) * iw;
        A1[c] = (sq[3 * (1 + c) + 2] - sq[3 * (1 + c)] * r2) * iw;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A0[c] = sq[c];
        A1[c] = sq[3 + c];
      }
    }
    const double A2[3] = {ip.ax, ip.ay, ip.az};
    double g0[3], g1[3], g2[3];
    cross3(A1, A2, g0);
    cross3(A2, A0, g1);
    cross3(A0, A1, g2);
    const double det = A0[0] * g0[0] + A0[1] * g0[1] + A0[2] * g0[2], inv = 1.0 / det;
    const int qu = q % ip.nqu, qv = q / ip.nqu;
    double* d = qd + (size_t)q * kShellQ;
    int e1 = 0, e2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = g0[c] * inv;
      d[3 + c] = g1[c] * inv;
      d[6 + c] = g2[c] * inv;
      e1 = max(e1, max(exp_field(d[c]), exp_field(d[3 + c])));
      e2 = max(e2, exp_field(d[6 + c]));
    }
    d[9] = ip.wU[(size_t)ex * ip.nqu + qu] * ip.wV[(size_t)ey * ip.nqv + qv] * fabs(det);
    d[10] = iw;
    d[11] = r1;
    d[12] = r2;
    atomicMax(&s_k[0], e1);
    atomicMax(&s_k[1], e2);
    atomicMax(&s_k[2], exp_field(d[9]));
  }
  __syncthreads();
  const int k1 = s_k[0] > 0 ? s_k[0] - 1023 : 0, k2 = s_k[1] > 0 ? s_k[1] - 1023 : 0;
  const int kq = s_k[2] > 0 ? s_k[2] - 1023 : 0;
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls, k = t % nls;
    const int qu = q % ip.nqu, qv = q / ip.nqu, lx = k % nlx, ly = k / nlx;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2 + 2 * lx;
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2 + 2 * ly;
    const double* d = qd + (size_t)q * kShellQ;
    float u0h, u0l, u1h, u1l, v0h, v0l, v1h, v1l;
    split_df_fast(tu[0], u0h, u0l);
    split_df_fast(tu[1], u1h, u1l);
    split_df_fast(tv[0], v0h, v0l);
    split_df_fast(tv[1], v1h, v1l);
    float Rh, Rl, R1h, R1l, R2h, R2l;
    df_prod(u0h, u0l, v0h, v0l, Rh, Rl);
    df_prod(u1h, u1l, v0h, v0l, R1h, R1l);
    df_prod(u0h, u0l, v1h, v1l, R2h, R2l);
    if (rat) {  // R = c N, R_,k = c (N_,k - N W_,k / W), c = w / W
      float ch, cl, rh, rl, th, tl;
      split_df_fast(ip.weights[(size_t)(fy + ly) * ip.nx + fx + lx] * d[10], ch, cl);
      split_df_fast(d[11], rh, rl);
      df_prod(Rh, Rl, -rh, -rl, th, tl);
      df_add(th, tl, R1h, R1l);
      df_norm(R1h, R1l);
      df_prod(R1h, R1l, ch, cl, R1h, R1l);
      split_df_fast(d[12], rh, rl);
      df_prod(Rh, Rl, -rh, -rl, th, tl);
      df_add(th, tl, R2h, R2l);
      df_norm(R2h, R2l);
      df_prod(R2h, R2l, ch, cl, R2h, R2l);
      df_prod(Rh, Rl, ch, cl, Rh, Rl);
    }
    float wh, wl;
    split_df_off(d[9], kq, wh, wl);
    float* f = phf + (size_t)t * 12;
    float* fw = pwf + (size_t)t * 12;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float ah, al, bh, bl, gh, gl, h, l;
      split_df_off(d[c], k1, ah, al);
      split_df_off(d[3 + c], k1, bh, bl);
      df_mul(ah, al, R1h, R1l, gh, gl);  // R_,1 g^0 + R_,2 g^1
      df_mac(bh, bl, R2h, R2l, gh, gl);
      df_norm(gh, gl);
      f[c] = gh;
      f[6 + c] = gl;
      df_prod(wh, wl, gh, gl, h, l);
      fw[c] = h;
      fw[6 + c] = l;
      split_df_off(d[6 + c], k2, ah, al);  // R g^2
      df_prod(Rh, Rl, ah, al, gh, gl);
      f[3 + c] = gh;
      f[9 + c] = gl;
      df_prod(wh, wl, gh, gl, h, l);
      fw[3 + c] = h;
      fw[9 + c] = l;
    }
  }
}

__global__ void __launch_bounds__(256) ka_shell(KaShellArgs a) {
  extern __shared__ double sm[];
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  const int e = blockIdx.x, ex = e % ip.nel_u, ey = e / ip.nel_u;
  const int nit = nqs * nls;
  float* phf = reinterpret_cast<float*>(sm);  // [item][12]: hi 6, lo 6
  float* pwf = phf + (size_t)nit * 12;
  double* qs = reinterpret_cast<double*>(pwf + (size_t)nit * 12);
  __shared__ int s_k[3];
  if (threadIdx.x < 3) s_k[threadIdx.x] = 0;
  __syncthreads();
  ka_shell_point_values(ip, ex, ey, phf, pwf, qs, s_k);
  const int k1 = s_k[0] > 0 ? s_k[0] - 1023 : 0, k2 = s_k[1] > 0 ? s_k[1] - 1023 : 0;
  const int kq = s_k[2] > 0 ? s_k[2] - 1023 : 0;
  __syncthreads();
  const int npl = nls * (nls + 1) / 2;
  double* out = a.EG + (size_t)e * npl * 36;
  for (int t = threadIdx.x; t < 4 * npl; t += blockDim.x) {
    const int blk = t / npl, pr = t % npl, al = blk >> 1, be = blk & 1;
    int li = 0, rem = pr;
    while (rem >= nls - li) {
      rem -= nls - li;
      ++li;
    }
    const int lj = li + rem;
    float sh[9], sl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sh[k] = sl[k] = 0.0f;
    for (int q = 0; q < nqs; ++q) {
      const float* A = pwf + ((size_t)q * nls + li) * 12;
      const float* B = phf + ((size_t)q * nls + lj) * 12;
      float ah[3], alo[3], bh[3], blo[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ah[k] = A[3 * al + k];
        alo[k] = A[6 + 3 * al + k];
        bh[k] = B[3 * be + k];
        blo[k] = B[6 + 3 * be + k];
      }
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) df_mac(ah[x], alo[x], bh[y], blo[y], sh[x * 3 + y], sl[x * 3 + y]);
    }
    const int sc = kq + (al ? k2 : k1) + (be ? k2 : k1);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float hs = __fadd_rn(sh[k], sl[k]);
      const float ls = __fsub_rn(sl[k], __fsub_rn(hs, sh[k]));
      long long b = __double_as_longlong(df_to_double(hs, ls));
      if (b & 0x7FFFFFFFFFFFFFFFll) b += (long long)sc * (1ll << 52);  // times 2^sc, exact
      out[(size_t)pr * 36 + blk * 9 + k] = __longlong_as_double(b);
    }
  }
}

// P of every configuration for a general extrusion: CTA per in-plane row i_s.
// The row's 6 x 6 Gram blocks are summed over the shared elements (fixed
// order), then P_(alpha beta)[c][d] = sum_(a,b)
// D_m[V(c,a)][V(d,b)] G_(alpha a)(beta b) (Eq. P) for every configuration m,
// into P[(m * nnz_s + pair) * 36 + blk * 9 + c * 3 + d]. The 9-term sums run
// in double-float on the FP32 pipes: each 3 x 3 Gram block is divided by a
// power of two 2^kg (largest entry in [1, 2)) and each configuration's D by
// 2^kE (host side), and P is scaled back by 2^(kE + kg), so any scale of
// geometry or material stays inside float range.
struct KpShellArgs {
  int nx, nel_u, nlx, nls, npl, ncfg;
  int64_t nnz_s;
  const int64_t* LSb;
  const int *lenX, *lenY, *loX, *loY, *eloX, *ehiX, *eloY, *ehiY, *firstU, *firstV;
  const double* EG;
  const float2* Edf;  // D_m[V(c,a)][V(d,b)] 2^-kE[m] as float pairs, [m][cd][ab]
  const int* kE;
  double* P;
  unsigned long long* pmax;  // largest |P| per block (bit patterns; positive doubles order as integers)
  int full;                  // 0: pairs with j_s >= i_s only (the combine reads the others transposed)
};

// SMEM_E: the configurations' D tables staged in shared memory (few configurations).
constexpr int kKpShellSmemCfg = 32;
// MONO: every D is monoclinic about z (D[I][J] = 0 for I < 4 <= J), so
// D[V(c,a)][V(d,b)] vanishes unless exactly-one-index-is-z holds for both
// (c, a) and (d, b) or for neither: 5 of the 9 terms per entry remain.
template <bool SMEM_E, bool MONO>
__global__ void __launch_bounds__(1024) kp_shell(KpShellArgs a) {
  extern __shared__ float2 sE[];  // the configurations' D tables (SMEM_E)
  __shared__ unsigned long long smax[4];
  if (threadIdx.x < 4) smax[threadIdx.x] = 0ull;
  if (SMEM_E)
    for (int k = threadIdx.x; k < a.ncfg * 81; k += blockDim.x) sE[k] = a.Edf[k];
  __syncthreads();
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  // thread per (k_s, block): the block's 9 Gram entries summed over the shared
  // elements (row-major element order), divided by 2^kg as float pairs in
  // registers, then its 9 entries of P for every configuration
  unsigned long long pm = 0ull;  // this thread's largest |P| (bit pattern: integer max, off the FP64 pipe)
  // P^ji_(alpha beta)[c][d] = P^ij_(beta alpha)[d][c]: unless asked for every pair,
  // only j_s >= i_s is formed, the neighbours from the row's own position on
  const int ks0 = a.full ? 0 : (iy - a.loY[iy]) * lx + (ix - a.loX[ix]);
  const int blk = threadIdx.x & 3;  // the same for every item of this thread (blockDim is a multiple of 32)
  for (int item = threadIdx.x; item < 4 * (ls - ks0); item += blockDim.x) {
    const int ks = ks0 + (item >> 2);
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
    const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
    const int blkT = (blk & 1) * 2 + (blk >> 1);  // the transposed block (beta, alpha)
    double g[9];
    bool first = true;  // the first element initialises the sums (one FP64 add fewer per entry)
    for (int ey = ey0; ey <= ey1; ++ey) {
      const int fy = a.firstV[ey];
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        const size_t e0 = ((size_t)ey * a.nel_u + ex) * a.npl;
        double v[9];
        if (li <= lj) {
          const double* src = a.EG + (e0 + upper_pair(li, lj, a.nls)) * 36 + blk * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) v[ab] = src[ab];
        } else {  // G^ji_(alpha a)(beta b) = G^ij_(beta b)(alpha a)
          const double* src = a.EG + (e0 + upper_pair(lj, li, a.nls)) * 36 + blkT * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) v[ab] = src[(ab % 3) * 3 + ab / 3];
        }
        if (first) {
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] = v[ab];
        } else {
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] += v[ab];
        }
        first = false;
      }
    }
    int e = 0;
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) e = max(e, exp_field(g[ab]));
    const int kg = e > 0 ? e - 1023 : 0;
    float gh[9], gl[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) split_df_off(g[ab], kg, gh[ab], gl[ab]);
    for (int m = 0; m < a.ncfg; ++m) {
      const float2* E = (SMEM_E ? sE : a.Edf) + (size_t)m * 81;
      const int sc = a.kE[m] + kg;
      double* out = a.P + ((size_t)m * a.nnz_s + ls0 + ks) * 36 + blk * 9;
#pragma unroll
      for (int cd = 0; cd < 9; ++cd) {
        float sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int ab = 0; ab < 9; ++ab) {
          const int c = cd / 3, d = cd % 3, aa = ab / 3, bb = ab % 3;
          if (MONO && (((c == 2) != (aa == 2)) != ((d == 2) != (bb == 2)))) continue;
          const float2 ee = SMEM_E ? E[cd * 9 + ab] : __ldg(E + cd * 9 + ab);
          df_mac(ee.x, ee.y, gh[ab], gl[ab], sh, sl);
        }
        const float hs = __fadd_rn(sh, sl);
        const float lsum = __fsub_rn(sl, __fsub_rn(hs, sh));
        long long b = __double_as_longlong(df_to_double(hs, lsum));
        if (b & 0x7FFFFFFFFFFFFFFFll) b += (long long)sc * (1ll << 52);  // exact
        out[cd] = __longlong_as_double(b);
        pm = max(pm, (unsigned long long)(b & 0x7FFFFFFFFFFFFFFFll));
      }
    }
  }
  // per block: the largest |P| over the CTA (lanes of one warp share blk modulo 4)
  for (int off = 16; off >= 4; off >>= 1) pm = max(pm, __shfl_xor_sync(0xffffffffu, pm, off));
  if ((threadIdx.x & 31) < 4) atomicMax(&smax[blk], pm);
  __syncthreads();
  if (threadIdx.x < 4) atomicMax(&a.pmax[threadIdx.x], smax[threadIdx.x]);
}

// K-a of a general extrusion in FP64: the output of ka_shell, with the point
// values of shell_points (u_1 = g1 = R_,1 g^0 + R_,2 g^1, u_2 = R g^2, w|DF|)
// and thread <-> (block (alpha, beta), unordered local pair), 9 FP64 fused
// multiply-adds per point: G_(alpha a)(beta b) = sum_q w|DF| u_alpha^li[a] u_beta^lj[b].
__global__ void __launch_bounds__(256) ka_shell64(KaShellArgs a) {
  extern __shared__ double sm[];
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  const int e = blockIdx.x, ex = e % ip.nel_u, ey = e / ip.nel_u;
  double* ph = sm;                              // [q][k][4]: g1 (3), R
  double* qs = ph + (size_t)nqs * nls * 4;      // [q][kShellQ]
  double* uu = qs + (size_t)nqs * kShellQ;      // [q][k][12]: u (6), w|DF| u (6)
  shell_points(ip, ex, ey, ph, qs);
  // u = (g1, R g^2) and its weighted copy, once per (point, function)
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls;
    const double* d = qs + (size_t)q * kShellQ;
    const double* f = ph + (size_t)t * 4;
    double* o = uu + (size_t)t * 12;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[k] = f[k];
      o[3 + k] = f[3] * d[6 + k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) o[6 + k] = d[9] * o[k];
  }
  __syncthreads();
  const int npl = nls * (nls + 1) / 2;
  double* out = a.EG + (size_t)e * npl * 36;
  for (int t = threadIdx.x; t < 4 * npl; t += blockDim.x) {
    const int blk = t / npl, pr = t % npl, al = blk >> 1, be = blk & 1;
    int li = 0, rem = pr;
    while (rem >= nls - li) {
      rem -= nls - li;
      ++li;
    }
    const int lj = li + rem;
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (int q = 0; q < nqs; ++q) {
      const double* ui = uu + ((size_t)q * nls + li) * 12 + 6 + 3 * al;  // w|DF| u_alpha^li
      const double* uj = uu + ((size_t)q * nls + lj) * 12 + 3 * be;      // u_beta^lj
      const double a0 = ui[0], a1 = ui[1], a2 = ui[2], b0 = uj[0], b1 = uj[1], b2 = uj[2];
      acc[0] = fma(a0, b0, acc[0]);
      acc[1] = fma(a0, b1, acc[1]);
      acc[2] = fma(a0, b2, acc[2]);
      acc[3] = fma(a1, b0, acc[3]);
      acc[4] = fma(a1, b1, acc[4]);
      acc[5] = fma(a1, b2, acc[5]);
      acc[6] = fma(a2, b0, acc[6]);
      acc[7] = fma(a2, b1, acc[7]);
      acc[8] = fma(a2, b2, acc[8]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) out[(size_t)pr * 36 + blk * 9 + k] = acc[k];
  }
}

// P of every configuration for a general extrusion in FP64: the output of
// kp_shell (same layout and pair set) with P_(alpha beta)[c][d] =
// sum_(a,b) D_m[V(c,a)][V(d,b)] G_(alpha a)(beta b) as FP64 fused multiply-adds
// (E = the configurations' cfgE tables, staged in shared memory when few).
template <bool SMEM_E, bool MONO>
__global__ void __launch_bounds__(1024) kp_shell64(KpShellArgs a, const double* __restrict__ cfgE) {
  extern __shared__ double sE64[];
  if (SMEM_E)
    for (int k = threadIdx.x; k < a.ncfg * 81; k += blockDim.x) sE64[k] = cfgE[k];
  __syncthreads();
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  const int ks0 = a.full ? 0 : (iy - a.loY[iy]) * lx + (ix - a.loX[ix]);
  const int blk = threadIdx.x & 3;
  for (int item = threadIdx.x; item < 4 * (ls - ks0); item += blockDim.x) {
    const int ks = ks0 + (item >> 2);
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
    const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
    const int blkT = (blk & 1) * 2 + (blk >> 1);
    double g[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) g[ab] = 0.0;
    for (int ey = ey0; ey <= ey1; ++ey) {
      const int fy = a.firstV[ey];
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        const size_t e0 = ((size_t)ey * a.nel_u + ex) * a.npl;
        if (li <= lj) {
          const double* src = a.EG + (e0 + upper_pair(li, lj, a.nls)) * 36 + blk * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] += src[ab];
        } else {
          const double* src = a.EG + (e0 + upper_pair(lj, li, a.nls)) * 36 + blkT * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] += src[(ab % 3) * 3 + ab / 3];
        }
      }
    }
    for (int m = 0; m < a.ncfg; ++m) {
      const double* E = (SMEM_E ? sE64 : cfgE) + (size_t)m * 81;
      double* out = a.P + ((size_t)m * a.nnz_s + ls0 + ks) * 36 + blk * 9;
#pragma unroll
      for (int cd = 0; cd < 9; ++cd) {
        double v = 0.0;
#pragma unroll
        for (int ab = 0; ab < 9; ++ab) {
          const int c = cd / 3, d = cd % 3, aa = ab / 3, bb = ab % 3;
          if (MONO && (((c == 2) != (aa == 2)) != ((d == 2) != (bb == 2)))) continue;
          v = fma(E[cd * 9 + ab], g[ab], v);
        }
        out[cd] = v;
      }
    }
  }
}

// The assembled 6 x 6 Gram blocks of every in-plane pair of a general extrusion
// (the adjoint's G): CTA per in-plane row, thread per (k_s, block), the block's
// 9 entries summed over the shared elements in row-major element order, FP64.
__global__ void __launch_bounds__(256) kg_shell(KpShellArgs a, double* __restrict__ G36) {
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  for (int item = threadIdx.x; item < 4 * ls; item += blockDim.x) {
    const int ks = item >> 2, blk = item & 3, blkT = (blk & 1) * 2 + (blk >> 1);
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
    const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
    double g[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) g[ab] = 0.0;
    for (int ey = ey0; ey <= ey1; ++ey) {
      const int fy = a.firstV[ey];
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        const size_t e0 = ((size_t)ey * a.nel_u + ex) * a.npl;
        if (li <= lj) {
          const double* src = a.EG + (e0 + upper_pair(li, lj, a.nls)) * 36 + blk * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] += src[ab];
        } else {  // G^ji_(alpha a)(beta b) = G^ij_(beta b)(alpha a)
          const double* src = a.EG + (e0 + upper_pair(lj, li, a.nls)) * 36 + blkT * 9;
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) g[ab] += src[(ab % 3) * 3 + ab / 3];
        }
      }
    }
    double* out = G36 + (ls0 + ks) * 36 + blk * 9;
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) out[ab] = g[ab];
  }
}

// The shells' adjoint Gram blocks rescaled in place: w = qs[blk] G_(blk)(ab)
// (the Q types enter divided by qs), gscale[ab] = a power of two at least
// max |w| over every pair and block, G = w / gscale[ab] (all exact) and its
// float pairs Gdf; both passes then accumulate in the same units.
__global__ void kg_shell_max(int64_t n36, const double* __restrict__ G36, double q0, double q1, double q2, double q3,
                             unsigned long long* __restrict__ gmax) {
  __shared__ unsigned long long smax[9];
  if (threadIdx.x < 9) smax[threadIdx.x] = 0ull;
  __syncthreads();
  const double qs[4] = {q0, q1, q2, q3};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n36; k += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(k % 36);
    atomicMax(&smax[e % 9], (unsigned long long)__double_as_longlong(fabs(qs[e / 9] * G36[k])));
  }
  __syncthreads();
  if (threadIdx.x < 9) atomicMax(&gmax[threadIdx.x], smax[threadIdx.x]);
}

__global__ void kg_shell_split(int64_t n36, double* __restrict__ G36, double q0, double q1, double q2,
                               double q3, const unsigned long long* __restrict__ gmax, float2* __restrict__ Gdf,
                               double* __restrict__ gscale) {
  __shared__ double inv[9];
  const double qs[4] = {q0, q1, q2, q3};
  if (threadIdx.x < 9) {
    const double m = __longlong_as_double((long long)gmax[threadIdx.x]);
    double sc = 1.0;
    if (m > 0.0 && m <= 1.7976931348623157e308) {
      int e = 0;
      frexp(m, &e);
      sc = ldexp(1.0, e);
    }
    inv[threadIdx.x] = 1.0 / sc;
    if (blockIdx.x == 0) gscale[threadIdx.x] = sc;
  }
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n36; k += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(k % 36);
    const double w = qs[e / 9] * G36[k] * inv[e % 9];
    G36[k] = w;
    float hi, lo;
    split_df(w, hi, lo);
    Gdf[k] = make_float2(hi, lo);
  }
}

// ---------------------------------------------------------------------------
// K-c: fused combine. One CTA per in-plane row i_s; thread <-> (c, k_s, d) of
// that row. The CTA first forms the row's G blocks (gathered from the element
// blocks, or loaded from an assembled G), the class Q vectors, and the CSR base
// of every (c, thickness occurrence). Each thread then forms its
// P_{m,ab}[c][d] from its G block and, for every thickness class u, evaluates
// slice_u = sum_terms sum_ab Q P once and stores it at every occurrence
// (i_t, k_t) of the class: one shared load and one 8-byte store per value.
// ---------------------------------------------------------------------------
struct KcArgs {
  int64_t ns, nnz_s;
  int nx, ncfg, ncls, nterms, nocc, gs_cap;
  const int64_t* LSb;
  const int *lenX, *lenY;
  const double* G;      // assembled G (nnz_s x 9), when not gathering
  // gathering from element blocks
  const double* EG;
  int nel_u, nlx, nls, npl;  // elements in u, local functions in x / per element, pairs per element
  const int *loX, *loY, *eloX, *ehiX, *eloY, *ehiY, *firstU, *firstV;
  const double* cfgE;
  const double* q;
  const int *cls_term_begin, *cls_terms, *cls_occ_begin, *term_rep;
  const int64_t* occ_A;
  const int *occ_lt, *occ_k, *occ_it;
  int it_lo, it_hi;     // thickness rows written (chunked output)
  int64_t out_offset;   // subtracted from every CSR position
  double* values;
  // streaming combine
  const int64_t* LTb;
  const int* pair_cls;
  int nchunk, slice_stride, nt, nslot_max, max_terms;
  const int *ck_it, *ck_term, *ck_nslot, *pair_slot;
  const int *ckt_slot, *ckt_cfg, *ckt_rep, *ckt_first;
  const float2* qdf;
  const int64_t* tp_A;
  const int *tp_lt, *tp_k;
  // double-float streaming combine
  const float2* cfgEdf;  // float pairs of cfgE
  int* flag;             // set when the FP64 pass must recompute
  int* emax;             // largest float exponent field of an entry
  int conditional;       // FP64 pass: run only if *flag != 0
  // general extrusion: P of every configuration, n_cfg x nnz_s x 36, and the
  // largest |P| of each block (11, 12, 21, 22) as bit patterns
  const double* shellP;
  const unsigned long long* shell_pmax;
  // monoclinic plates: per-kind source terms and the copies of the other slots
  const int *ck_sterm, *ck_nblk, *cks_slot, *cks_cfg, *cks_rep, *cks_first;
  const int *ck_copy, *ckc_dst, *ckc_src;
  int max_copies;
  // per in-plane pair, the element blocks its G sums (the plan's pair-sum table; null if not built)
  const int *gsum_begin, *gsum_off;
};

// Entries (c, d) of a monoclinic 3 x 3 block by kind: block (c and d both
// in-plane or both z: Q_11, Q_22) first, then off (Q_12, Q_21). A thread of the
// combine's slice arithmetic takes entry kBlkC/D[g] (g < 5) or kOffC/D[g - 5]
// for in-plane neighbour k_s, so that most warps hold one kind.
__constant__ int kKindC[9] = {0, 0, 1, 1, 2, 0, 1, 2, 2};
__constant__ int kKindD[9] = {0, 1, 0, 1, 2, 2, 2, 0, 1};


// G_ab of the in-plane pair (i_s, k_s-th neighbour j_s): the sum over the shared
// elements, row-major in (ey, ex), of the element blocks of K-a. Loads go out
// four at a time before their adds; missing entries of a group add an exact
// zero. The same order everywhere it is formed (kg_rows, kcs_row), so every
// path that assembles a row's G gets the same bits.
__device__ __forceinline__ double gram_pair_sum(const KcArgs& a, int ix, int iy, int lx, int ks, int ab) {
  const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
  const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
  const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
  const int ba = (ab % 3) * 3 + ab / 3;
  const int nex = ex1 - ex0 + 1, ne = nex * (ey1 - ey0 + 1);
  double acc = 0.0;
  for (int q0 = 0; q0 < ne; q0 += 4) {
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j;
      v[j] = 0.0;
      if (q < ne) {
        const int ey = ey0 + q / nex, ex = ex0 + q % nex;
        const int fy = a.firstV[ey], fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        const size_t ep = ((size_t)ey * a.nel_u + ex) * a.npl;
        v[j] = li <= lj ? a.EG[(ep + upper_pair(li, lj, a.nls)) * 9 + ab]
                        : a.EG[(ep + upper_pair(lj, li, a.nls)) * 9 + ba];
      }
    }
    acc = ((acc + v[0]) + v[1]) + v[2];
    acc = acc + v[3];
  }
  return acc;
}

// gram_pair_sum from the pair's precomputed list of element-block positions
// (same blocks, same order, same grouping of the adds: the same bits).
__device__ __forceinline__ double gram_pair_sum_tab(const double* __restrict__ EG, const int* __restrict__ gb,
                                                    const int* __restrict__ go, int64_t pr, int ab) {
  const int ba = (ab % 3) * 3 + ab / 3;
  const int b0 = __ldg(gb + pr), b1 = __ldg(gb + pr + 1);
  double acc = 0.0;
  for (int q0 = b0; q0 < b1; q0 += 4) {
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = 0.0;
      if (q0 + j < b1) {
        const int o = __ldg(go + q0 + j);
        v[j] = EG[(o >> 1) + ((o & 1) ? ba : ab)];
      }
    }
    acc = ((acc + v[0]) + v[1]) + v[2];
    acc = acc + v[3];
  }
  return acc;
}

// P of a general extrusion for entry (c, d) of the in-plane pair (i_s, k_s-th
// neighbour j_s): pairs with j_s >= i_s hold it (blocks at 0, 9, 18, 27); the
// others read the mirror pair transposed, P^ij_(alpha beta)[c][d] =
// P^ji_(beta alpha)[d][c], so blocks 12 and 21 trade places.
struct ShellPRef {
  const double* p;  // entry of block 11 of configuration 0
  int o12, o21;     // offsets of blocks 12 and 21
};
__device__ __forceinline__ ShellPRef shell_p_ref(const KcArgs& a, int64_t is, int ix, int iy, int lx, int64_t ls0,
                                                 int ks, int c, int d) {
  const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
  const int64_t js = (int64_t)jy * a.nx + jx;
  if (js >= is) return ShellPRef{a.shellP + (size_t)(ls0 + ks) * 36 + c * 3 + d, 9, 18};
  const int ksT = (iy - a.loY[jy]) * a.lenX[jx] + (ix - a.loX[jx]);
  return ShellPRef{a.shellP + (size_t)(a.LSb[js] + ksT) * 36 + d * 3 + c, 18, 9};
}

template <bool MONO, bool CHUNKED, bool GATHER, bool SHELL = false>
__global__ void __launch_bounds__(1024, 2) kc_combine(KcArgs a) {
  static_assert(!(SHELL && MONO), "a general extrusion couples every block");
  extern __shared__ double sm[];
  constexpr int NP = MONO ? 2 : 4;
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix];
  const int ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  const int nthr = blockDim.x, tid = threadIdx.x;
  // shared layout
  double* Gs = sm;                                         // 9 * ls (max)
  double* Ps = Gs + a.gs_cap;                              // ncfg * NP * nthr
  double* Qs = Ps + (size_t)a.ncfg * NP * nthr;            // nterms * 4
  int64_t* base3 = reinterpret_cast<int64_t*>(Qs + (size_t)a.nterms * 4);  // 3 * nocc
  int* tb = reinterpret_cast<int*>(base3 + 3 * (size_t)a.nocc);            // ncls + 1
  int* ob = tb + (a.ncls + 1);                             // ncls + 1
  int* tm = ob + (a.ncls + 1);                             // nterms
  if (SHELL) {
  } else if (GATHER) {
    for (int item = tid; item < 9 * ls; item += nthr) {
      const int ks = item / 9, ab = item % 9;
      const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
      const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
      const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
      const int ba = (ab % 3) * 3 + ab / 3;
      double acc = 0.0;
      for (int ey = ey0; ey <= ey1; ++ey) {
        const int fy = a.firstV[ey];
        for (int ex = ex0; ex <= ex1; ++ex) {
          const int fx = a.firstU[ex];
          const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
          const size_t ep = ((size_t)ey * a.nel_u + ex) * a.npl;
          if (li <= lj)
            acc += a.EG[(ep + upper_pair(li, lj, a.nls)) * 9 + ab];
          else
            acc += a.EG[(ep + upper_pair(lj, li, a.nls)) * 9 + ba];
        }
      }
      Gs[item] = acc;
    }
  } else {
    for (int k = tid; k < 9 * ls; k += nthr) Gs[k] = a.G[ls0 * 9 + k];
  }
  for (int k = tid; k < a.nterms; k += nthr) {
    const int m = a.cls_terms[k];
    tm[k] = m;
    const double* src = a.q + ((size_t)a.term_rep[k] * a.ncfg + m) * 4;
    Qs[4 * k + 0] = src[0];
    Qs[4 * k + 1] = src[1];
    Qs[4 * k + 2] = src[2];
    Qs[4 * k + 3] = src[3];
  }
  // CSR base of (c, occurrence o): row_ptr(i_t, i_s, c) + 3 k_t len_s, minus the output offset
  for (int o = tid; o < a.nocc; o += nthr) {
    const int64_t A = a.occ_A[o];
    const int64_t lt = a.occ_lt[o], kt = a.occ_k[o];
    const bool keep = !CHUNKED || (a.occ_it[o] >= a.it_lo && a.occ_it[o] < a.it_hi);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      base3[(size_t)c * a.nocc + o] =
          keep ? A + lt * (9 * ls0 + 3 * (int64_t)c * ls) + kt * 3 * (int64_t)ls - a.out_offset : (int64_t)-1;
  }
  for (int k = tid; k <= a.ncls; k += nthr) {
    tb[k] = a.cls_term_begin[k];
    ob[k] = a.cls_occ_begin[k];
  }
  __syncthreads();
  const int item = tid;
  if (item >= 9 * ls) return;
  const int c = item / (3 * ls), rem = item % (3 * ls), ks = rem / 3, d = rem % 3;
  const double* g = Gs + ks * 9;
  const int cd = c * 3 + d;
  // P for every configuration, into shared memory (indexed by the class terms)
  const bool block_type = ((c == 2) == (d == 2));
  ShellPRef pr{nullptr, 9, 18};
  if (SHELL) pr = shell_p_ref(a, is, ix, iy, lx, ls0, ks, c, d);
  for (int m = 0; m < a.ncfg; ++m) {
    const double* E = a.cfgE + (size_t)m * 81 + cd * 9;
    const double* Pp = SHELL ? pr.p + (size_t)m * a.nnz_s * 36 : nullptr;
    const double p11 = SHELL ? Pp[0] : E[0] * g[0] + E[1] * g[1] + E[3] * g[3] + E[4] * g[4];
    const double p12 = SHELL ? Pp[pr.o12] : E[2] * g[2] + E[5] * g[5];
    const double p21 = SHELL ? Pp[pr.o21] : E[6] * g[6] + E[7] * g[7];
    const double p22 = SHELL ? Pp[27] : E[8] * g[8];
    if (MONO) {
      Ps[(m * 2 + 0) * nthr + tid] = block_type ? p11 : p12;
      Ps[(m * 2 + 1) * nthr + tid] = block_type ? p22 : p21;
    } else {
      Ps[(m * 4 + 0) * nthr + tid] = p11;
      Ps[(m * 4 + 1) * nthr + tid] = p12;
      Ps[(m * 4 + 2) * nthr + tid] = p21;
      Ps[(m * 4 + 3) * nthr + tid] = p22;
    }
  }
  const int offa = block_type ? 0 : 1, offb = block_type ? 3 : 2;
  const int64_t* B = base3 + (size_t)c * a.nocc;
  double* out = a.values + (3 * ks + d);
  for (int u = 0; u < a.ncls; ++u) {
    double v = 0.0;
    for (int k = tb[u]; k < tb[u + 1]; ++k) {
      const int m = tm[k];
      if (MONO) {
        v += Qs[4 * k + offa] * Ps[(m * 2 + 0) * nthr + tid] + Qs[4 * k + offb] * Ps[(m * 2 + 1) * nthr + tid];
      } else {
        v += Qs[4 * k + 0] * Ps[(m * 4 + 0) * nthr + tid] + Qs[4 * k + 1] * Ps[(m * 4 + 1) * nthr + tid] +
             Qs[4 * k + 2] * Ps[(m * 4 + 2) * nthr + tid] + Qs[4 * k + 3] * Ps[(m * 4 + 3) * nthr + tid];
      }
    }
    const int o1 = ob[u + 1];
#pragma unroll 4
    for (int o = ob[u]; o < o1; ++o) {
      const int64_t b = B[o];
      if (CHUNKED && b < 0) continue;
      out[b] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// K-c, streaming form (used when a row's class slices fit in shared memory):
// one CTA per in-plane row i_s (threads = 9 max len_s rounded up to warps: 448
// for cubic rows), as many CTAs per SM as 64 registers per thread allow (two
// for cubic rows). The double-float pass of the plan's opt-in arithmetic, the
// FP64 fallback when kc_ws's two buffers do not fit, and the batches' rows. Phase 1 forms the
// row's G blocks (gathered from the element blocks); each thread (c, k_s, d)
// forms the P_{m,ab}[c][d] it needs per configuration and accumulates
// slice_u = sum Q P for every class u in shared memory. Phase 2 writes the
// row's share of the CSR values in address order: for each thickness row i_t
// the 3 rows c, each of len_t segments of 3 len_s values, are contiguous; each
// warp copies the three segments of one thickness pair, issuing all of a
// segment's shared loads before its global stores. The other CTA on the SM
// computes while this one stores.
//
// DF = true: phase 1 in double-float arithmetic on the FP32 pipes (G, D and Q
// split into float pairs; products to about 2^-47, two-sums), slices turned
// into doubles by df_to_double. A slice that is not finite, or a matrix whose
// largest entry is below 2^-60, sets the flag; the FP64 form (DF = false,
// conditional) then recomputes every row on the same stream.
// ---------------------------------------------------------------------------
constexpr int kSegUnroll = 6;  // 32 * 6 >= 3 * len_s for rows of at most 512 / 9 neighbours
constexpr int kKcMinExp = 127 - 60;  // float exponent field of 2^-60

// P_{m,ab}[c][d] for one configuration as float pairs: MONO gives (pa, pb)
// (the two products a monoclinic block needs), otherwise p11, p12, p21, p22.
__device__ __forceinline__ void df_dot(const float2* __restrict__ E, const float* gh, const float* gl, int k0, int k1,
                                       int k2, int k3, int n, float& h, float& l) {
  const int ks[4] = {k0, k1, k2, k3};
  h = 0.0f;
  l = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < n) {
      const float2 e = E[ks[j]];
      float p, q;
      df_mul(e.x, e.y, gh[ks[j]], gl[ks[j]], p, q);
      df_add(p, q, h, l);
    }
  }
  const float hs = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(hs, h));
  h = hs;
}

// One in-plane row i_s of the streaming combine (phases 0 to 2 for every
// chunk of thickness rows). `sm` is the CTA's dynamic shared memory; emax and
// bad accumulate the double-float pass's range checks.
template <bool MONO, bool CHUNKED, bool DF, bool SHELL = false>
// pcache (FP64 monoclinic rows only, may be NULL): 2 * n_cfg * blockDim.x doubles
// of this CTA's own, which receive the thread's P (p_a, p_b) of every
// configuration once per row; the chunks read them back instead of forming P
// again (a row of an uneven stack meets all configurations in each of its chunks).
__device__ __forceinline__ void kcs_row(const KcArgs& a, int64_t is, double* sm, int& emax, bool& bad,
                                        double* pcache = nullptr) {
  static_assert(!(SHELL && MONO), "a general extrusion couples every block");
  const int nthr = blockDim.x, tid = threadIdx.x;
  double* slices = sm;  // slots x stride (the G row first)
  double* sQ = sm + (size_t)a.nslot_max * a.slice_stride;                  // chunk terms: Q
  int* sSlot = reinterpret_cast<int*>(sQ + 4 * (size_t)a.max_terms);       // slot
  int* sFirst = sSlot + a.max_terms;                                       // first term of its slot
  int* sCfg = sFirst + a.max_terms;                                        // configuration
  int* sCopyDst = sCfg + a.max_terms;                                      // FP64, monoclinic: copied slots
  int* sCopySrc = sCopyDst + a.max_copies;                                 // ... and their source slots
  // FP64 on a monoclinic plate: the per-kind source terms and slot copies of kc_ws
  constexpr bool SPLIT = MONO && !DF && !SHELL;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix];
  const int ls = lx * a.lenY[iy];
  const int n9 = 9 * ls;
  const int64_t ls0 = a.LSb[is];
  // phase 0: the row's G blocks into slices[0 .. 9 ls) (a general extrusion reads P instead);
  // the double-float pass reads the pair-sum table (the FP64 form, register-bound in
  // batches, keeps the index arithmetic: fewer registers live)
  for (int item = tid; item < (SHELL ? 0 : n9); item += nthr)
    slices[item] = (DF && a.gsum_off) ? gram_pair_sum_tab(a.EG, a.gsum_begin, a.gsum_off, ls0 + item / 9, item % 9)
                                      : gram_pair_sum(a, ix, iy, lx, item / 9, item % 9);
  __syncthreads();
  // entries grouped by kind (SPLIT): block kind (5 ls entries) first, then off
  // kind (4 ls); where the CTA has room the block kind is padded to whole warps,
  // so that no warp runs both kinds' term loops (entry e of thread tid)
  bool active = tid < n9;
  int e = tid;
  if (SPLIT) {
    const int nb = 5 * ls, pb = (nb + 31) & ~31;
    if (pb + 4 * ls <= nthr) {
      active = tid < pb ? tid < nb : tid - pb < 4 * ls;
      e = tid < pb ? tid : nb + (tid - pb);
    }
  }
  int c = 0, ks = 0, d = 0;
  double g[9];
  float gh[9], gl[9];
  if (active) {
    if (SPLIT) {
      const int gk = e / ls;
      ks = e - gk * ls;
      c = kKindC[gk];
      d = kKindD[gk];
    } else {
      c = tid / (3 * ls);
      const int rem = tid % (3 * ls);
      ks = rem / 3;
      d = rem % 3;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      g[k] = SHELL ? 0.0 : slices[ks * 9 + k];
      if (DF && !SHELL) split_df(g[k], gh[k], gl[k]);
    }
  }
  __syncthreads();  // the G row is in registers; its space is reused by the slices
  const int item = active ? c * 3 * ls + 3 * ks + d : tid;  // the entry's place in a slice (output order)
  const int cd = c * 3 + d;
  const bool block_type = ((c == 2) == (d == 2));
  const int offa = block_type ? 0 : 1, offb = block_type ? 3 : 2;
  const int seg_len = 3 * ls;
  // general extrusion, double-float pass: block j of P enters divided by 2^ps[j]
  // (its largest entry in [1, 2)) and Q_j multiplied by it (exact), so that the
  // float pairs hold blocks of very different magnitude (P_22 / P_11 ~ L^2).
  // (blocks 12 and 21 share one scale: over all pairs max |P_12| = max |P_21|,
  // and only pairs j_s >= i_s are formed)
  int ps[4] = {0, 0, 0, 0};
  ShellPRef pref{nullptr, 9, 18};
  if (SHELL) {
    if (active) pref = shell_p_ref(a, is, ix, iy, lx, ls0, ks, c, d);
    if (DF) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int jj = (j == 1 || j == 2) ? 3 - j : j;
        const unsigned long long bits = max(a.shell_pmax[j], a.shell_pmax[jj]);
        const double mx = __longlong_as_double((long long)bits);
        ps[j] = mx > 0.0 ? exp_field(mx) - 1023 : 0;
      }
    }
  }
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  const bool use_pcache = SPLIT && pcache != nullptr;
  if (use_pcache && active) {
    for (int m = 0; m < a.ncfg; ++m) {  // the same fused multiply-adds as below, stored once
      const double* E = a.cfgE + (size_t)m * 81 + cd * 9;
      double pa, pb;
      if (block_type) {
        pa = fma(E[4], g[4], fma(E[3], g[3], fma(E[1], g[1], E[0] * g[0])));
        pb = E[8] * g[8];
      } else {
        pa = fma(E[5], g[5], E[2] * g[2]);
        pb = fma(E[7], g[7], E[6] * g[6]);
      }
      pcache[(size_t)(2 * m) * nthr + tid] = pa;
      pcache[(size_t)(2 * m + 1) * nthr + tid] = pb;
    }
  }
  for (int ch = 0; ch < a.nchunk; ++ch) {
    int it0 = a.ck_it[ch], it1 = a.ck_it[ch + 1];
    if (CHUNKED) {
      it0 = max(it0, a.it_lo);
      it1 = min(it1, a.it_hi);
      if (it0 >= it1) continue;  // the same for every thread
    }
    // the chunk's terms into shared memory
    const int tb = SPLIT ? a.ck_sterm[ch] : a.ck_term[ch];
    const int nterm = (SPLIT ? a.ck_sterm[ch + 1] : a.ck_term[ch + 1]) - tb;
    const int nblk = SPLIT ? a.ck_nblk[ch] : 0;
    const int cb = SPLIT ? a.ck_copy[ch] : 0, ncopy = SPLIT ? a.ck_copy[ch + 1] - cb : 0;
    for (int k = tid; k < ncopy; k += nthr) {
      sCopyDst[k] = a.ckc_dst[cb + k];
      sCopySrc[k] = a.ckc_src[cb + k];
    }
    for (int k = tid; k < nterm; k += nthr) {
      const int t = tb + k, m = SPLIT ? a.cks_cfg[t] : a.ckt_cfg[t];
      const size_t qi = ((size_t)(SPLIT ? a.cks_rep[t] : a.ckt_rep[t]) * a.ncfg + m) * 4;
      if (DF) {
        float2* q2 = reinterpret_cast<float2*>(sQ + 4 * (size_t)k);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 v = a.qdf[qi + j];
          q2[j] = SHELL ? make_float2(ldexpf(v.x, ps[j]), ldexpf(v.y, ps[j])) : v;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) sQ[4 * (size_t)k + j] = a.q[qi + j];
      }
      sSlot[k] = SPLIT ? a.cks_slot[t] : a.ckt_slot[t];
      sFirst[k] = SPLIT ? a.cks_first[t] : a.ckt_first[t];
      sCfg[k] = m;
    }
    __syncthreads();
    // phase 1: slice of every class of the chunk (terms sorted by configuration)
    if (active) {
      const int t1 = nterm;
      int cur = -1;
      if (DF) {
        float ah = 0.0f, al = 0.0f, bh = 0.0f, bl = 0.0f, ch_ = 0.0f, cl = 0.0f, dh = 0.0f, dl = 0.0f;
        for (int t = 0; t < t1; ++t) {
          const int m = sCfg[t];
          if (m != cur) {
            cur = m;
            const float2* E = a.cfgEdf + (size_t)m * 81 + cd * 9;
            if (SHELL) {
              const double* Pp = pref.p + (size_t)m * a.nnz_s * 36;
              split_df_off(Pp[0], ps[0], ah, al);
              split_df_off(Pp[pref.o12], ps[1], bh, bl);
              split_df_off(Pp[pref.o21], ps[2], ch_, cl);
              split_df_off(Pp[27], ps[3], dh, dl);
            } else if (MONO) {
              if (block_type) {
                df_dot(E, gh, gl, 0, 1, 3, 4, 4, ah, al);
                df_dot(E, gh, gl, 8, 8, 8, 8, 1, bh, bl);
              } else {
                df_dot(E, gh, gl, 2, 5, 0, 0, 2, ah, al);
                df_dot(E, gh, gl, 6, 7, 0, 0, 2, bh, bl);
              }
            } else {
              df_dot(E, gh, gl, 0, 1, 3, 4, 4, ah, al);
              df_dot(E, gh, gl, 2, 5, 0, 0, 2, bh, bl);
              df_dot(E, gh, gl, 6, 7, 0, 0, 2, ch_, cl);
              df_dot(E, gh, gl, 8, 8, 8, 8, 1, dh, dl);
            }
          }
          const float2* q2 = reinterpret_cast<const float2*>(sQ + 4 * (size_t)t);
          float vh, vl, p, e;
          if (MONO) {
            const float2 qa = q2[offa], qb = q2[offb];
            df_mul(qa.x, qa.y, ah, al, vh, vl);
            df_mul(qb.x, qb.y, bh, bl, p, e);
            df_add(p, e, vh, vl);
          } else {
            df_mul(q2[0].x, q2[0].y, ah, al, vh, vl);
            df_mul(q2[1].x, q2[1].y, bh, bl, p, e);
            df_add(p, e, vh, vl);
            df_mul(q2[2].x, q2[2].y, ch_, cl, p, e);
            df_add(p, e, vh, vl);
            df_mul(q2[3].x, q2[3].y, dh, dl, p, e);
            df_add(p, e, vh, vl);
          }
          float2* dst = reinterpret_cast<float2*>(slices + (size_t)sSlot[t] * a.slice_stride + item);
          if (!sFirst[t]) {
            const float2 o = *dst;
            df_add(o.x, o.y, vh, vl);
          }
          *dst = make_float2(vh, vl);
        }
        // float pairs -> doubles, in place (each thread its own column)
        const int ns_ = a.ck_nslot[ch];
        for (int u = 0; u < ns_; ++u) {
          double* dst = slices + (size_t)u * a.slice_stride + item;
          const float2 v = *reinterpret_cast<const float2*>(dst);
          const float hs = __fadd_rn(v.x, v.y);
          const float lsum = __fsub_rn(v.y, __fsub_rn(hs, v.x));
          const int ef = (int)((__float_as_uint(hs) >> 23) & 0xFFu);
          bad |= (ef == 255);
          emax = max(emax, ef);
          *dst = df_to_double(hs, lsum);
        }
      } else {
        double pa = 0.0, pb = 0.0, p11 = 0.0, p12 = 0.0, p21 = 0.0, p22 = 0.0;
        const int t_begin = (SPLIT && !block_type) ? nblk : 0;
        const int t_end = (SPLIT && block_type) ? nblk : t1;
        for (int t = t_begin; t < t_end; ++t) {
          const int m = sCfg[t];
          if (m != cur) {
            cur = m;
            const double* E = a.cfgE + (size_t)m * 81 + cd * 9;
            if (SHELL) {
              const double* Pp = pref.p + (size_t)m * a.nnz_s * 36;
              p11 = Pp[0];
              p12 = Pp[pref.o12];
              p21 = Pp[pref.o21];
              p22 = Pp[27];
            } else if (use_pcache) {
              pa = pcache[(size_t)(2 * m) * nthr + tid];
              pb = pcache[(size_t)(2 * m + 1) * nthr + tid];
            } else if (MONO) {  // the fused multiply-adds of kc_ws, in its order (bitwise equal results)
              if (block_type) {
                pa = fma(E[4], g[4], fma(E[3], g[3], fma(E[1], g[1], E[0] * g[0])));
                pb = E[8] * g[8];
              } else {
                pa = fma(E[5], g[5], E[2] * g[2]);
                pb = fma(E[7], g[7], E[6] * g[6]);
              }
            } else {
              p11 = fma(E[4], g[4], fma(E[3], g[3], fma(E[1], g[1], E[0] * g[0])));
              p12 = fma(E[5], g[5], E[2] * g[2]);
              p21 = fma(E[7], g[7], E[6] * g[6]);
              p22 = E[8] * g[8];
            }
          }
          const double* Q = sQ + 4 * (size_t)t;
          double* dst = slices + (size_t)sSlot[t] * a.slice_stride + item;
          double v = sFirst[t] ? 0.0 : *dst;
          if (MONO) {
            v = fma(Q[offa], pa, v);
            v = fma(Q[offb], pb, v);
          } else {
            v = fma(Q[0], p11, v);
            v = fma(Q[1], p12, v);
            v = fma(Q[2], p21, v);
            v = fma(Q[3], p22, v);
          }
          *dst = v;
        }
        if (SPLIT) {  // slots that share this kind's Q terms with a source slot
          const int kind = block_type ? 0 : 1;
          for (int q = 0; q < ncopy; ++q) {
            const int dk = sCopyDst[q];
            if ((dk & 1) == kind)
              slices[(size_t)(dk >> 1) * a.slice_stride + item] = slices[(size_t)sCopySrc[q] * a.slice_stride + item];
          }
        }
      }
    }
    __syncthreads();
    // phase 2: the chunk's thickness pairs (i_t, k_t) in address order, one
    // warp per pair. Row (i_t, i_s, c) holds len_t segments of 3 len_s
    // values; the pair's three segments (c = 0, 1, 2) sit one row apart. Each
    // copy issues all of its shared loads before its global stores.
    const int64_t p_end = a.LTb[it1];
    for (int64_t pr = a.LTb[it0] + warp; pr < p_end; pr += nwarps) {
      const int64_t A = a.tp_A[pr];
      const int lt = a.tp_lt[pr], kt = a.tp_k[pr], u = a.pair_slot[pr];
      const double* src = slices + (size_t)u * a.slice_stride;
      double* dst = a.values + (A + (int64_t)lt * 9 * ls0 + (int64_t)kt * seg_len - a.out_offset);
      const int64_t row_step = (int64_t)lt * seg_len;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        double v[kSegUnroll];
#pragma unroll
        for (int j = 0; j < kSegUnroll; ++j) v[j] = (lane + 32 * j < seg_len) ? src[cc * seg_len + lane + 32 * j] : 0.0;
#pragma unroll
        for (int j = 0; j < kSegUnroll; ++j)
          if (lane + 32 * j < seg_len) dst[cc * row_step + lane + 32 * j] = v[j];
      }
    }
    __syncthreads();  // the slices are rewritten by the next chunk or row
  }
}

template <bool MONO, bool CHUNKED, bool DF, bool SHELL = false>
__global__ void __maxnreg__(64) kc_stream(KcArgs a) {
  // FP64 pass after a double-float one: only if a slice was not finite or no entry reached 2^-60
  if (!DF && a.conditional && *a.flag == 0 && *a.emax >= kKcMinExp) return;
  extern __shared__ double sm[];
  int emax = 0;
  bool bad = false;
  for (int64_t is = blockIdx.x; is < a.ns; is += gridDim.x) kcs_row<MONO, CHUNKED, DF, SHELL>(a, is, sm, emax, bad);
  if (DF) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(a.emax, emax);
      if (any_bad) atomicOr(a.flag, 1);
    }
  }
}

// ---------------------------------------------------------------------------
// K-c in FP64, warp-specialised streaming form. One persistent CTA per SM
// takes the work units (in-plane row i_s, thickness chunk) of rows
// blockIdx.x, blockIdx.x + gridDim.x, ... Its first nct threads (the compute
// group, thread (c, k_s, d) of the row as in kcs_row) load the row's
// assembled G (kg_rows), form P_{m,ab}[c][d] per configuration (Eq. P for a homogeneous ply) and the
// class slices sum_m sum_ab Q_{m,ab} P_{m,ab} (Eq. Km_2) with FP64 fused
// multiply-adds into one of two shared-memory buffers, while the other warps
// (the copy group) write the previous unit's share of the CSR values from the
// other buffer in address order. The FP64 pipe and the HBM writes are thus
// busy at the same time instead of in alternating phases. Hand-offs use
// hardware named barriers: FULL[b] (compute arrives, copy waits) when buffer b
// holds a unit's slices, EMPTY[b] (copy arrives, compute waits) when the copy
// group has read it; both groups walk the same unit sequence, so every
// barrier is met exactly as often by both sides.
// ---------------------------------------------------------------------------
constexpr int kBarCompute = 1, kBarFull = 2, kBarEmpty = 4;
// (the non-.aligned forms: threads of a warp may reach them after divergent code)
__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n) {
  asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// the chunk's thickness rows, clipped to the rows written (CHUNKED output); false if none
template <bool CHUNKED>
__device__ __forceinline__ bool kcw_chunk(const KcArgs& a, int ch, int& it0, int& it1) {
  it0 = a.ck_it[ch];
  it1 = a.ck_it[ch + 1];
  if (CHUNKED) {
    it0 = max(it0, a.it_lo);
    it1 = min(it1, a.it_hi);
  }
  return it0 < it1;
}

// The assembled in-plane Gram blocks of every in-plane pair, G_ab(i_s, k_s) =
// sum over the shared elements (fixed row-major element order) of the element
// blocks of K-a, into G[(LSb[i_s] + k_s) * 9 + ab]: CTA per in-plane row,
// thread per (k_s, ab). FP64 sums, the order of the combine's own gather; the
// blocks' positions come from the plan's per-pair table (gb, go) when it was
// built, else from the index arithmetic of gram_pair_sum.
__global__ void __launch_bounds__(512, 4) kg_rows(KcArgs a, double* __restrict__ G, const int* __restrict__ gb,
                                                  const int* __restrict__ go) {
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], n9 = 9 * lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  for (int it = threadIdx.x; it < n9; it += blockDim.x) {
    const double acc = go ? gram_pair_sum_tab(a.EG, gb, go, ls0 + it / 9, it % 9)
                          : gram_pair_sum(a, ix, iy, lx, it / 9, it % 9);
    G[ls0 * 9 + it] = acc;
  }
}

// Copies the thickness pairs of one unit (pairs p_begin .. p_begin + npairs - 1
// of row i_s, slices in S) into the CSR values, one warp per pair: the pair's
// three segments (c = 0, 1, 2) of 3 len_s values, one CSR row apart. Pairs are
// handed out by the shared counter *next, so any number of warps can join; a
// warp takes its next pair (and loads that pair's table entries) before it
// copies the current one.
template <int U>
__device__ __forceinline__ void kcw_copy_pairs(const KcArgs& a, const double* S, int* next, int64_t p_begin,
                                               int npairs, int64_t ls0, int seg_len, int lane) {
  auto take = [&]() {
    int q = 0;
    if (lane == 0) q = atomicAdd(next, 1);
    return __shfl_sync(0xffffffffu, q, 0);
  };
  int q = take();
  int64_t A = 0;
  int lt = 0, kt = 0, u = 0;
  if (q < npairs) {
    A = __ldg(a.tp_A + p_begin + q);
    lt = __ldg(a.tp_lt + p_begin + q);
    kt = __ldg(a.tp_k + p_begin + q);
    u = __ldg(a.pair_slot + p_begin + q);
  }
  while (q < npairs) {
    const int qn = take();
    int64_t An = 0;
    int ltn = 0, ktn = 0, un = 0;
    if (qn < npairs) {
      An = __ldg(a.tp_A + p_begin + qn);
      ltn = __ldg(a.tp_lt + p_begin + qn);
      ktn = __ldg(a.tp_k + p_begin + qn);
      un = __ldg(a.pair_slot + p_begin + qn);
    }
    const double* src = S + (size_t)u * a.slice_stride;
    double* dst = a.values + (A + (int64_t)lt * 9 * ls0 + (int64_t)kt * seg_len - a.out_offset);
    const int64_t row_step = (int64_t)lt * seg_len;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      double v[U];  // U * 32 >= 3 len_s of the plan's longest row
#pragma unroll
      for (int j = 0; j < U; ++j) v[j] = (lane + 32 * j < seg_len) ? src[cc * seg_len + lane + 32 * j] : 0.0;
#pragma unroll
      for (int j = 0; j < U; ++j)
        if (lane + 32 * j < seg_len) dst[cc * row_step + lane + 32 * j] = v[j];
    }
    q = qn;
    A = An;
    lt = ltn;
    kt = ktn;
    u = un;
  }
}

template <bool MONO, bool CHUNKED, bool SHELL, int U>
__global__ void __launch_bounds__(896, 1) kc_ws(KcArgs a, int nct) {
  static_assert(!(SHELL && MONO), "a general extrusion couples every block");
  extern __shared__ double sm[];
  const int tid = threadIdx.x, nall = blockDim.x;
  const size_t buf_elems = (size_t)a.nslot_max * a.slice_stride;
  double* sG = sm + 2 * buf_elems;                                     // the row's G blocks (9 per neighbour)
  double* sQ = sG + a.slice_stride;                                    // chunk terms: Q
  int2* sMeta = reinterpret_cast<int2*>(sQ + 4 * (size_t)a.max_terms);  // (2 slot + first, configuration)
  int* sCopyDst = reinterpret_cast<int*>(sMeta + a.max_terms);           // monoclinic: copied slots (2 slot + kind)
  int* sCopySrc = sCopyDst + a.max_copies;                               // ... and their source slots
  int* sNext = sCopySrc + a.max_copies;                                  // next pair of each buffer's unit
  if (tid < 2) sNext[tid] = 0;
  __syncthreads();  // the only CTA-wide barrier: the groups part here
  int nch_eff = 0;
  for (int ch = 0; ch < a.nchunk; ++ch) {
    int it0, it1;
    nch_eff += kcw_chunk<CHUNKED>(a, ch, it0, it1) ? 1 : 0;
  }
  const int64_t nrows = blockIdx.x < a.ns ? (a.ns - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nunits = nrows * nch_eff;
  if (tid < nct) {
    // ---------------- compute group ----------------
    int k = 0, loaded = -1, nblk = 0, ncopy = 0;
    double gpre = 0.0;  // this thread's G entry of the next row (prefetched)
    const int lane = tid & 31;
    // the previous unit, whose copy the compute warps join once their own slices are done
    int prev_b = -1, prev_np = 0, prev_seg = 0;
    int64_t prev_p0 = 0, prev_ls0 = 0;
    for (int64_t is = blockIdx.x; is < a.ns; is += gridDim.x) {
      const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
      const int lx = a.lenX[ix];
      const int ls = lx * a.lenY[iy];
      const int n9 = 9 * ls;
      const int64_t ls0 = a.LSb[is];
      const bool active = tid < n9;
      int c = 0, ks = 0, d = 0;
      if (active && MONO) {  // entries grouped by kind: block first, then off
        const int g = tid / ls;
        ks = tid - g * ls;
        c = kKindC[g];
        d = kKindD[g];
      } else if (active) {
        c = tid / (3 * ls);
        const int rem = tid % (3 * ls);
        ks = rem / 3;
        d = rem % 3;
      }
      const int item = active ? c * 3 * ls + 3 * ks + d : tid;  // the entry's place in a slice (output order)
      const int cd = c * 3 + d;
      const bool block_type = ((c == 2) == (d == 2));
      const int offa = block_type ? 0 : 1, offb = block_type ? 3 : 2;
      ShellPRef pref{nullptr, 9, 18};
      if (SHELL && active) pref = shell_p_ref(a, is, ix, iy, lx, ls0, ks, c, d);
      bool first_unit_of_row = true;
      for (int ch = 0; ch < a.nchunk; ++ch) {
        int it0, it1;
        if (!kcw_chunk<CHUNKED>(a, ch, it0, it1)) continue;
        const int b = k & 1;
        double* S = sm + (size_t)b * buf_elems;
        if (k >= 2) named_bar_sync(kBarEmpty + b, nall);  // the copy group has read buffer b
        if (!SHELL && first_unit_of_row) {
          // phase 0: the row's assembled G blocks (kg_rows) into sG, after every
          // thread has formed its last P from the previous row's; the entry of
          // this thread was loaded during the previous row (one load per thread,
          // n9 <= nct), and the next row's entry is requested right after
          if (k > 0) named_bar_sync(kBarCompute, nct);
          if (k == 0 && tid < n9) gpre = a.G[ls0 * 9 + tid];
          if (tid < n9) sG[tid] = gpre;
          named_bar_sync(kBarCompute, nct);
          const int64_t nx_is = is + gridDim.x;
          if (nx_is < a.ns) {
            const int nix = (int)(nx_is % a.nx), niy = (int)(nx_is / a.nx);
            if (tid < 9 * a.lenX[nix] * a.lenY[niy]) gpre = a.G[a.LSb[nx_is] * 9 + tid];
          }
        }
        first_unit_of_row = false;
        // the chunk's terms (loaded once when the plan has one chunk); monoclinic
        // plates: the block kind's source terms, the off kind's, and the copies
        const int tb = MONO ? a.ck_sterm[ch] : a.ck_term[ch];
        const int nterm = (MONO ? a.ck_sterm[ch + 1] : a.ck_term[ch + 1]) - tb;
        if (loaded != ch) {
          if (loaded >= 0) named_bar_sync(kBarCompute, nct);  // nobody still reads the previous chunk's terms
          for (int q = tid; q < nterm; q += nct) {
            const int t = tb + q, m = MONO ? a.cks_cfg[t] : a.ckt_cfg[t];
            const size_t qi = ((size_t)(MONO ? a.cks_rep[t] : a.ckt_rep[t]) * a.ncfg + m) * 4;
#pragma unroll
            for (int j = 0; j < 4; ++j) sQ[4 * (size_t)q + j] = a.q[qi + j];
            sMeta[q] = MONO ? make_int2(2 * a.cks_slot[t] + (a.cks_first[t] ? 1 : 0), m)
                            : make_int2(2 * a.ckt_slot[t] + (a.ckt_first[t] ? 1 : 0), m);
          }
          if (MONO) {
            nblk = a.ck_nblk[ch];
            const int cb = a.ck_copy[ch];
            ncopy = a.ck_copy[ch + 1] - cb;
            for (int q = tid; q < ncopy; q += nct) {
              sCopyDst[q] = a.ckc_dst[cb + q];
              sCopySrc[q] = a.ckc_src[cb + q];
            }
          }
          named_bar_sync(kBarCompute, nct);
          loaded = ch;
        }
        // phase 1: the slice of every class of the chunk, FP64
        if (active) {
          const double* g = sG + ks * 9;
          int cur = -1;
          double pa = 0.0, pb = 0.0, p11 = 0.0, p12 = 0.0, p21 = 0.0, p22 = 0.0;
          const int t_begin = (MONO && !block_type) ? nblk : 0;
          const int t_end = (MONO && block_type) ? nblk : nterm;
          for (int t = t_begin; t < t_end; ++t) {
            const int2 meta = sMeta[t];
            const int m = meta.y;
            if (m != cur) {
              cur = m;
              if (SHELL) {
                const double* Pp = pref.p + (size_t)m * a.nnz_s * 36;
                p11 = Pp[0];
                p12 = Pp[pref.o12];
                p21 = Pp[pref.o21];
                p22 = Pp[27];
              } else {
                const double* E = a.cfgE + (size_t)m * 81 + cd * 9;
                if (MONO) {
                  if (block_type) {
                    pa = fma(E[4], g[4], fma(E[3], g[3], fma(E[1], g[1], E[0] * g[0])));
                    pb = E[8] * g[8];
                  } else {
                    pa = fma(E[5], g[5], E[2] * g[2]);
                    pb = fma(E[7], g[7], E[6] * g[6]);
                  }
                } else {
                  p11 = fma(E[4], g[4], fma(E[3], g[3], fma(E[1], g[1], E[0] * g[0])));
                  p12 = fma(E[5], g[5], E[2] * g[2]);
                  p21 = fma(E[7], g[7], E[6] * g[6]);
                  p22 = E[8] * g[8];
                }
              }
            }
            const double* Q = sQ + 4 * (size_t)t;
            double* dst = S + (size_t)(meta.x >> 1) * a.slice_stride + item;
            double v = (meta.x & 1) ? 0.0 : *dst;
            if (MONO) {
              v = fma(Q[offa], pa, v);
              v = fma(Q[offb], pb, v);
            } else {
              v = fma(Q[0], p11, v);
              v = fma(Q[1], p12, v);
              v = fma(Q[2], p21, v);
              v = fma(Q[3], p22, v);
            }
            *dst = v;
          }
          if (MONO) {  // slots that share this kind's Q terms with a source slot
            const int kind = block_type ? 0 : 1;
            for (int q = 0; q < ncopy; ++q) {
              const int dk = sCopyDst[q];
              if ((dk & 1) == kind) S[(size_t)(dk >> 1) * a.slice_stride + item] = S[(size_t)sCopySrc[q] * a.slice_stride + item];
            }
          }
        }
        if (tid == 0) sNext[b] = 0;  // nobody takes pairs of buffer b until FULL[b] completes
        __threadfence_block();
        named_bar_arrive(kBarFull + b, nall);  // buffer b holds the unit's slices
        // join the copy of the previous unit, whose buffer the next unit reuses
        if (prev_b >= 0)
          kcw_copy_pairs<U>(a, sm + (size_t)prev_b * buf_elems, sNext + prev_b, prev_p0, prev_np, prev_ls0, prev_seg, lane);
        prev_b = b;
        prev_p0 = a.LTb[it0];
        prev_np = (int)(a.LTb[it1] - a.LTb[it0]);
        prev_ls0 = ls0;
        prev_seg = 3 * ls;
        ++k;
      }
    }
    if (prev_b >= 0) {  // the last unit: every compute thread's slices are visible after the barrier
      named_bar_sync(kBarCompute, nct);
      kcw_copy_pairs<U>(a, sm + (size_t)prev_b * buf_elems, sNext + prev_b, prev_p0, prev_np, prev_ls0, prev_seg, lane);
    }
  } else {
    // ---------------- copy group ----------------
    const int lane = tid & 31;
    int64_t k = 0;
    for (int64_t is = blockIdx.x; is < a.ns; is += gridDim.x) {
      const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
      const int ls = a.lenX[ix] * a.lenY[iy];
      const int seg_len = 3 * ls;
      const int64_t ls0 = a.LSb[is];
      for (int ch = 0; ch < a.nchunk; ++ch) {
        int it0, it1;
        if (!kcw_chunk<CHUNKED>(a, ch, it0, it1)) continue;
        const int b = (int)(k & 1);
        const double* S = sm + (size_t)b * buf_elems;
        named_bar_sync(kBarFull + b, nall);
        kcw_copy_pairs<U>(a, S, sNext + b, a.LTb[it0], (int)(a.LTb[it1] - a.LTb[it0]), ls0, seg_len, lane);
        if (k + 2 < nunits) {
          __threadfence_block();
          named_bar_arrive(kBarEmpty + b, nall);  // buffer b may be overwritten
        }
        ++k;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K-a in FP64 (single launch): one CTA per in-plane element, the same output
// as ka_local. Point values (Eq. gradient: g = (dR/dx, dR/dy, R) and w|DF| g
// at every Gauss point) by inplane_points, then thread <-> unordered local
// pair (li <= lj): G_ab = sum_q (w|DF| g_a^li)(q) g_b^lj(q), 9 FP64 fused
// multiply-adds per point, into EG[(e * npl + pair) * 9 + ab].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ka_elem64(const KaLocalArgs& a, int e, double* sm) {
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  double* phi = sm;
  double* phiw = phi + (size_t)nqs * nls * 3;
  double* qd = phiw + (size_t)nqs * nls * 3;
  const int ex = e % ip.nel_u, ey = e / ip.nel_u;
  inplane_points(ip, ex, ey, phi, phiw, qd);
  const int npl = nls * (nls + 1) / 2;
  double* out = a.EG + (size_t)e * npl * 9;
  for (int t = threadIdx.x; t < npl; t += blockDim.x) {
    int li = 0, rem = t;
    while (rem >= nls - li) {
      rem -= nls - li;
      ++li;
    }
    const int lj = li + rem;
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    for (int q = 0; q < nqs; ++q) {
      const double* A = phiw + ((size_t)q * nls + li) * 3;
      const double* B = phi + ((size_t)q * nls + lj) * 3;
      const double a0 = A[0], a1 = A[1], a2 = A[2], b0 = B[0], b1 = B[1], b2 = B[2];
      acc[0] = fma(a0, b0, acc[0]);
      acc[1] = fma(a0, b1, acc[1]);
      acc[2] = fma(a0, b2, acc[2]);
      acc[3] = fma(a1, b0, acc[3]);
      acc[4] = fma(a1, b1, acc[4]);
      acc[5] = fma(a1, b2, acc[5]);
      acc[6] = fma(a2, b0, acc[6]);
      acc[7] = fma(a2, b1, acc[7]);
      acc[8] = fma(a2, b2, acc[8]);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) out[(size_t)t * 9 + q] = acc[q];
  }
}

__global__ void __launch_bounds__(256) ka_local64(KaLocalArgs a) {
  extern __shared__ double sm[];
  ka_elem64(a, blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// K-d: standard element-by-element quadrature (Section 2.4). One CTA per 3D
// element of one colour; thread <-> pairs (li <= lj) of local 3D functions.
// For each ply piece of the element: Gram of the 3D gradients over the piece's
// points, contracted with D of the piece's ply; both blocks of the pair are
// scattered into the CSR values.
// ---------------------------------------------------------------------------
struct KdArgs {
  InplaneArgs ip;
  const int* elems;
  int nel_v, nqt, q1;
  int64_t ns, nnz_s;
  const int *loX, *lenX, *loY, *lenY, *loT, *lenT, *firstT;
  const int64_t *LSb, *LTb;
  const int *piece_begin, *piece_cfg;
  const double *tabT, *wT, *cfgE;
  double* values;
};

__device__ __forceinline__ int64_t csr_pos(const KdArgs& a, int it, int64_t is, int c, int jt, int64_t js) {
  const int ix = (int)(is % a.ip.nx), iy = (int)(is / a.ip.nx);
  const int jx = (int)(js % a.ip.nx), jy = (int)(js / a.ip.nx);
  const int64_t lt = a.LTb[it + 1] - a.LTb[it];
  const int64_t ls = (int64_t)a.lenX[ix] * a.lenY[iy];
  const int64_t ks = (int64_t)(jy - a.loY[iy]) * a.lenX[ix] + (jx - a.loX[ix]);
  const int64_t kt = jt - a.loT[it];
  return 9 * a.LTb[it] * a.nnz_s + 9 * lt * a.LSb[is] + 3 * c * lt * ls + (kt * ls + ks) * 3;
}

// SHELL: a general extrusion, whose 3D gradients T g1 + T' R g^2 come from
// shell_points (planar: (g_x T, g_y T, R T')).
template <bool SHELL>
__global__ void __launch_bounds__(256) kd_standard(KdArgs a) {
  extern __shared__ double sm[];
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  constexpr int NV = SHELL ? 4 : 3, NQ = SHELL ? kShellQ : 8, WQ = SHELL ? 9 : 4;
  double* phi = sm;
  double* qd = phi + (size_t)nqs * nls * NV;
  const int e3 = a.elems[blockIdx.x];
  const int ex = e3 % ip.nel_u, ey = (e3 / ip.nel_u) % a.nel_v, et = e3 / (ip.nel_u * a.nel_v);
  if (SHELL)
    shell_points(ip, ex, ey, phi, qd);
  else
    inplane_points(ip, ex, ey, phi, nullptr, qd);
  const int nl = nls * a.q1;
  const int npairs = nl * (nl + 1) / 2;
  const int fx = ip.firstU[ex], fy = ip.firstV[ey], ft = a.firstT[et];
  const int pc0 = a.piece_begin[et], pc1 = a.piece_begin[et + 1];
  // the element's thickness values weighted by their Gauss weights, per
  // (piece, point, function): w_t T and w_t T' (one product fewer per 3D point
  // and pair side than weighting inside the point loop)
  double* tw = qd + (size_t)nqs * NQ;
  const int ntw = (pc1 - pc0) * a.nqt * a.q1;
  for (int k = threadIdx.x; k < ntw; k += blockDim.x) {
    const int pcg = k / a.q1;  // (pc - pc0) * nqt + g
    const double w = a.wT[(size_t)pc0 * a.nqt + pcg];
    const double* tb = a.tabT + ((size_t)pc0 * a.nqt * a.q1 + k) * 2;
    tw[2 * k] = w * tb[0];
    tw[2 * k + 1] = w * tb[1];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
    int li = 0, rem = t;
    while (rem >= nl - li) {
      rem -= nl - li;
      ++li;
    }
    const int lj = li + rem;
    const int lti = li / nls, lsi = li % nls, ltj = lj / nls, lsj = lj % nls;
    double K[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) K[k] = 0.0;
    for (int pc = pc0; pc < pc1; ++pc) {
      double acc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = 0.0;
      for (int qs = 0; qs < nqs; ++qs) {
        const double* A = phi + ((size_t)qs * nls + lsi) * NV;
        const double* B = phi + ((size_t)qs * nls + lsj) * NV;
        const double* dq = qd + (size_t)qs * NQ;
        const double ws = dq[WQ];
        const double wa0 = ws * A[0], wa1 = ws * A[1], wa2 = ws * A[2];  // the in-plane weight, once per point
        for (int g = 0; g < a.nqt; ++g) {
          const double* tt = tw + ((size_t)(pc - pc0) * a.nqt + g) * a.q1 * 2;  // weighted thickness values
          const double* tb = a.tabT + ((size_t)pc * a.nqt + g) * a.q1 * 2;
          const double Ti = tt[2 * lti], dTi = tt[2 * lti + 1], Tj = tb[2 * ltj], dTj = tb[2 * ltj + 1];
          double a0, a1, a2, b0, b1, b2;
          if (SHELL) {
            const double si = dTi * A[3], sj = dTj * B[3];
            a0 = ws * fma(Ti, A[0], si * dq[6]);
            a1 = ws * fma(Ti, A[1], si * dq[7]);
            a2 = ws * fma(Ti, A[2], si * dq[8]);
            b0 = fma(Tj, B[0], sj * dq[6]);
            b1 = fma(Tj, B[1], sj * dq[7]);
            b2 = fma(Tj, B[2], sj * dq[8]);
          } else {
            a0 = wa0 * Ti;
            a1 = wa1 * Ti;
            a2 = wa2 * dTi;
            b0 = B[0] * Tj;
            b1 = B[1] * Tj;
            b2 = B[2] * dTj;
          }
          acc[0] += a0 * b0;
          acc[1] += a0 * b1;
          acc[2] += a0 * b2;
          acc[3] += a1 * b0;
          acc[4] += a1 * b1;
          acc[5] += a1 * b2;
          acc[6] += a2 * b0;
          acc[7] += a2 * b1;
          acc[8] += a2 * b2;
        }
      }
      const double* E = a.cfgE + (size_t)a.piece_cfg[pc] * 81;
#pragma unroll
      for (int cd = 0; cd < 9; ++cd) {
        double s = 0.0;
#pragma unroll
        for (int ab = 0; ab < 9; ++ab) s += E[cd * 9 + ab] * acc[ab];
        K[cd] += s;
      }
    }
    const int it = ft + lti, jt = ft + ltj;
    const int64_t is = (int64_t)(fy + lsi / nlx) * ip.nx + fx + lsi % nlx;
    const int64_t js = (int64_t)(fy + lsj / nlx) * ip.nx + fx + lsj % nlx;
    for (int c = 0; c < 3; ++c) {
      const int64_t pos = csr_pos(a, it, is, c, jt, js);
      for (int d = 0; d < 3; ++d) a.values[pos + d] += K[c * 3 + d];
    }
    if (li != lj) {
      for (int d = 0; d < 3; ++d) {
        const int64_t pos = csr_pos(a, jt, js, d, it, is);
        for (int c = 0; c < 3; ++c) a.values[pos + c] += K[c * 3 + d];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Device set-up
// ---------------------------------------------------------------------------

// The element blocks each in-plane pair's G sums, in the order of the row
// gathers (shared elements row-major in (ey, ex)): per pair, 2 x (position of
// the block in EG) + 1 when the pair is read transposed (li > lj). False when
// a position or the table length would not fit an int (kg_rows then finds the
// blocks itself).
static bool pair_sum_table(const Plan& P, std::vector<int>& gb, std::vector<int>& go) {
  const int nlx = P.u.p + 1, nls = ka_nls(P), npl = ka_npl(P);
  if ((int64_t)P.u.nel * P.v.nel * npl * 9 * 2 >= (int64_t)INT32_MAX) return false;
  auto upper = [](int a, int b, int n) { return a * n - a * (a - 1) / 2 + (b - a); };
  gb.assign((size_t)P.nnz_s + 1, 0);
  go.clear();
  for (int64_t is = 0; is < P.ns; ++is) {
    const int ix = (int)(is % P.u.n), iy = (int)(is / P.u.n);
    const int lx = P.u.len[ix], ly = P.v.len[iy];
    for (int ks = 0; ks < lx * ly; ++ks) {
      const int jx = P.u.lo[ix] + ks % lx, jy = P.v.lo[iy] + ks / lx;
      const int ex0 = std::max(P.u.elo[ix], P.u.elo[jx]), ex1 = std::min(P.u.ehi[ix], P.u.ehi[jx]);
      const int ey0 = std::max(P.v.elo[iy], P.v.elo[jy]), ey1 = std::min(P.v.ehi[iy], P.v.ehi[jy]);
      for (int ey = ey0; ey <= ey1; ++ey)
        for (int ex = ex0; ex <= ex1; ++ex) {
          const int fy = P.v.first[ey], fx = P.u.first[ex];
          const int li = (iy - fy) * nlx + (ix - fx), lj = (jy - fy) * nlx + (jx - fx);
          const int64_t e = (int64_t)ey * P.u.nel + ex;
          const int64_t pos = (e * npl + (li <= lj ? upper(li, lj, nls) : upper(lj, li, nls))) * 9;
          go.push_back((int)(2 * pos + (li <= lj ? 0 : 1)));
        }
      if (go.size() >= (size_t)INT32_MAX) return false;
      gb[(size_t)(P.LSb[is] + ks) + 1] = (int)go.size();
    }
  }
  return true;
}
static lam_status ensure_device(Plan& P) {
  int cur = 0;
  LAM_CUDA(cudaGetDevice(&cur));
  if (P.dev && cur != P.device_id) {
    set_error("plan lives on device %d, current device is %d", P.device_id, cur);
    return LAM_ERR_INVALID_ARG;
  }
  lam_status st = LAM_OK;
#define UP(list, dst, src)                                   \
  do {                                                       \
    if ((st = upload(P, (list), &(dst), (src))) != LAM_OK) { \
      free_device(P);                                        \
      return st;                                             \
    }                                                        \
  } while (0)
  if (!P.dev) {
    Device* D = new Device();
    P.dev = D;
    P.device_id = cur;
    P.cfg_dirty = true;
    auto& L = D->allocs;
    UP(L, D->tabU, P.tabU);
    UP(L, D->tabV, P.tabV);
    UP(L, D->wU, P.wU);
    UP(L, D->wV, P.wV);
    UP(L, D->firstU, P.u.first);
    UP(L, D->firstV, P.v.first);
    UP(L, D->loX, P.u.lo);
    UP(L, D->lenX, P.u.len);
    UP(L, D->loY, P.v.lo);
    UP(L, D->lenY, P.v.len);
    UP(L, D->ctrl, P.ctrl);
    if (P.shell) UP(L, D->ctrl3, P.ctrl3);
    if (!P.weights.empty()) UP(L, D->weights, P.weights);
    UP(L, D->LSb, P.LSb);
    UP(L, D->col2_elem, P.col2_elem);
    UP(L, D->loT, P.t.lo);
    UP(L, D->lenT, P.t.len);
    UP(L, D->firstT, P.t.first);
    UP(L, D->LTb, P.LTb);
    UP(L, D->tabT, P.tabT);
    UP(L, D->wT, P.wT);
    UP(L, D->piece_begin, P.piece_begin);
    UP(L, D->tp_row, P.tp_row);
    UP(L, D->tp_col, P.tp_col);
    UP(L, D->tp_e0, P.tp_e0);
    UP(L, D->tp_e1, P.tp_e1);
    UP(L, D->tp_A, P.tp_A);
    UP(L, D->tp_lt, P.tp_lt);
    UP(L, D->tp_k, P.tp_k);
    UP(L, D->col3_elem, P.col3_elem);
    UP(L, D->eloX, P.u.elo);
    UP(L, D->ehiX, P.u.ehi);
    UP(L, D->eloY, P.v.elo);
    UP(L, D->ehiY, P.v.ehi);
    if ((st = alloc_dev(L, &D->EG, (size_t)P.u.nel * P.v.nel * 9 * ka_npl(P))) != LAM_OK) {
      free_device(P);
      return st;
    }
    if ((st = alloc_dev(L, &D->Grow, (size_t)P.nnz_s * 9)) != LAM_OK) {
      free_device(P);
      return st;
    }
    if (!P.shell) {
      std::vector<int> gb, go;
      if (pair_sum_table(P, gb, go)) {
        UP(L, D->gsum_begin, gb);
        UP(L, D->gsum_off, go);
      }
    }
    double* fl = nullptr;
    if ((st = alloc_dev(L, &fl, 1)) != LAM_OK) {
      free_device(P);
      return st;
    }
    D->kc_flag = reinterpret_cast<int*>(fl);
    LAM_CUDA(cudaDeviceGetAttribute(&D->n_sm, cudaDevAttrMultiProcessorCount, cur));
    LAM_CUDA(cudaDeviceGetAttribute(&D->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cur));
  }
  if (P.cfg_dirty) {
    Device* D = P.dev;
    LAM_CUDA(cudaDeviceSynchronize());  // no launch may still read the old tables
    free_cfg_tables(*D);
    auto& L = D->cfg_allocs;
    std::vector<int> pcfg(P.pieces.size());
    for (size_t k = 0; k < P.pieces.size(); ++k) pcfg[k] = P.pieces[k].cfg;
    UP(L, D->piece_cfg, pcfg);
    UP(L, D->cls_term_begin, P.cls_term_begin);
    UP(L, D->cls_terms, P.cls_terms);
    UP(L, D->cls_occ_begin, P.cls_occ_begin);
    std::vector<int> trep(P.cls_terms.size());
    for (int u = 0; u < P.ncls; ++u)
      for (int k = P.cls_term_begin[u]; k < P.cls_term_begin[u + 1]; ++k) trep[k] = P.cls_rep[u];
    UP(L, D->term_rep, trep);
    UP(L, D->occ_A, P.occ_A);
    UP(L, D->occ_lt, P.occ_lt);
    UP(L, D->occ_k, P.occ_k);
    UP(L, D->occ_it, P.occ_it);
    UP(L, D->cfgE, P.cfgE);
    UP(L, D->cfgCb, P.cfgCb);
    std::vector<float> edf(P.cfgE.size() * 2);
    for (size_t k = 0; k < P.cfgE.size(); ++k) {
      const float h = (float)P.cfgE[k];
      edf[2 * k] = h;
      edf[2 * k + 1] = (float)(P.cfgE[k] - (double)h);
    }
    float* edf_dev = nullptr;
    UP(L, edf_dev, edf);
    D->cfgEdf = reinterpret_cast<float2*>(edf_dev);
    if (P.shell) {  // D of every configuration divided by a power of two (largest entry in [1, 2))
      const int nc = (int)(P.cfgE.size() / 81);
      std::vector<int> kE(nc, 0);
      std::vector<float> sedf(P.cfgE.size() * 2);
      for (int m = 0; m < nc; ++m) {
        double mx = 0.0;
        for (int k = 0; k < 81; ++k) mx = std::max(mx, std::fabs(P.cfgE[(size_t)m * 81 + k]));
        if (mx > 0.0) kE[m] = std::ilogb(mx);
        for (int k = 0; k < 81; ++k) {
          const double e = std::ldexp(P.cfgE[(size_t)m * 81 + k], -kE[m]);
          const float h = (float)e;
          sedf[2 * ((size_t)m * 81 + k)] = h;
          sedf[2 * ((size_t)m * 81 + k) + 1] = (float)(e - (double)h);
        }
      }
      float* sedf_dev = nullptr;
      UP(L, sedf_dev, sedf);
      D->shell_Edf = reinterpret_cast<float2*>(sedf_dev);
      UP(L, D->shell_kE, kE);
    }
    UP(L, D->pair_cls, P.pair_cls);
    UP(L, D->ck_it, P.ck_it);
    UP(L, D->ck_term, P.ck_term);
    UP(L, D->ck_nslot, P.ck_nslot);
    UP(L, D->pair_slot, P.pair_slot);
    UP(L, D->ckt_slot, P.ckt_slot);
    UP(L, D->ckt_cfg, P.ckt_cfg);
    UP(L, D->ckt_rep, P.ckt_rep);
    UP(L, D->ckt_first, P.ckt_first);
    UP(L, D->ck_sterm, P.ck_sterm);
    UP(L, D->ck_nblk, P.ck_nblk);
    UP(L, D->cks_slot, P.cks_slot);
    UP(L, D->cks_cfg, P.cks_cfg);
    UP(L, D->cks_rep, P.cks_rep);
    UP(L, D->cks_first, P.cks_first);
    UP(L, D->ck_copy, P.ck_copy);
    UP(L, D->ckc_dst, P.ckc_dst);
    UP(L, D->ckc_src, P.ckc_src);
    UP(L, D->ply_M, P.ply_M);
    UP(L, D->ply_dM, P.ply_dM);
    UP(L, D->mat_C, P.mat_C);
    UP(L, D->ply_mat, P.ply_mat);
    if ((st = alloc_dev(L, &D->q, (size_t)P.nnz_t * P.cfg_mat.size() * 4)) != LAM_OK) {
      free_device(P);
      return st;
    }
    double* qdf = nullptr;
    if ((st = alloc_dev(L, &qdf, (size_t)P.nnz_t * P.cfg_mat.size() * 4)) != LAM_OK) {
      free_device(P);
      return st;
    }
    D->qdf = reinterpret_cast<float2*>(qdf);
    D->q_valid = false;
    P.cfg_dirty = false;
  }
#undef UP
  return LAM_OK;
}

static lam_status check_limits(const Plan& P) {
  if (P.nt > 65535) {
    set_error("more than 65535 thickness functions are not supported");
    return LAM_ERR_UNSUPPORTED;
  }
  if (9 * max_len_s(P) > 1024) {
    set_error("in-plane rows with more than %d neighbours are not supported by the combine kernel", 1024 / 9);
    return LAM_ERR_UNSUPPORTED;
  }
  // the class-major combine's tables matter where it runs (a general extrusion
  // takes the streaming form whenever that fits, and has no allocation-free path)
  const bool class_major = !(P.shell && use_stream(P));
  if ((class_major && kc_smem(P) > 200 * 1024) || ka_smem(P) > 200 * 1024 || kd_smem(P) > 200 * 1024 ||
      (P.shell && ka_shell_smem(P) > 200 * 1024) ||
      (P.shell && P.arith == LAM_ARITH_FP64 && ka_shell64_smem(P) > 200 * 1024)) {
    set_error("plan tables exceed the shared-memory budget of the kernels");
    return LAM_ERR_UNSUPPORTED;
  }
  return LAM_OK;
}

static InplaneArgs inplane_args(const Plan& P) {
  const Device& D = *P.dev;
  InplaneArgs ip;
  ip.nx = P.u.n;
  ip.nel_u = P.u.nel;
  ip.pu = P.u.p;
  ip.pv = P.v.p;
  ip.nqu = P.nqu;
  ip.nqv = P.nqv;
  ip.tabU = D.tabU;
  ip.tabV = D.tabV;
  ip.wU = D.wU;
  ip.wV = D.wV;
  ip.ctrl = D.ctrl;
  ip.weights = D.weights;
  ip.firstU = D.firstU;
  ip.firstV = D.firstV;
  ip.ctrl3 = D.ctrl3;
  ip.ax = P.extrusion[0];
  ip.ay = P.extrusion[1];
  ip.az = P.extrusion[2];
  return ip;
}

static KcArgs kc_args(const Plan& P, double* values) {
  const Device& D = *P.dev;
  KcArgs k{};
  k.ns = P.ns;
  k.nnz_s = P.nnz_s;
  k.nx = P.u.n;
  k.ncfg = (int)P.cfg_mat.size();
  k.ncls = P.ncls;
  k.nterms = (int)P.cls_terms.size();
  k.nocc = (int)P.nnz_t;
  k.gs_cap = kc_gs_cap(P);
  k.LSb = D.LSb;
  k.lenX = D.lenX;
  k.lenY = D.lenY;
  k.G = nullptr;
  k.EG = D.EG;
  k.nel_u = P.u.nel;
  k.nlx = P.u.p + 1;
  k.nls = ka_nls(P);
  k.npl = ka_npl(P);
  k.loX = D.loX;
  k.loY = D.loY;
  k.eloX = D.eloX;
  k.ehiX = D.ehiX;
  k.eloY = D.eloY;
  k.ehiY = D.ehiY;
  k.firstU = D.firstU;
  k.firstV = D.firstV;
  k.cfgE = D.cfgE;
  k.q = D.q;
  k.cls_term_begin = D.cls_term_begin;
  k.cls_terms = D.cls_terms;
  k.cls_occ_begin = D.cls_occ_begin;
  k.term_rep = D.term_rep;
  k.occ_A = D.occ_A;
  k.occ_lt = D.occ_lt;
  k.occ_k = D.occ_k;
  k.occ_it = D.occ_it;
  k.it_lo = 0;
  k.it_hi = (int)P.nt;
  k.out_offset = 0;
  k.values = values;
  k.LTb = D.LTb;
  k.pair_cls = D.pair_cls;
  k.nchunk = (int)P.ck_nslot.size();
  k.nslot_max = 1;
  for (int v : P.ck_nslot) k.nslot_max = std::max(k.nslot_max, v);
  k.max_terms = kcs_max_terms(P);
  k.ck_it = D.ck_it;
  k.ck_term = D.ck_term;
  k.ck_nslot = D.ck_nslot;
  k.pair_slot = D.pair_slot;
  k.ckt_slot = D.ckt_slot;
  k.ckt_cfg = D.ckt_cfg;
  k.ckt_rep = D.ckt_rep;
  k.ckt_first = D.ckt_first;
  k.qdf = D.qdf;
  k.slice_stride = kcs_stride(P);
  k.nt = (int)P.nt;
  k.tp_A = D.tp_A;
  k.tp_lt = D.tp_lt;
  k.tp_k = D.tp_k;
  k.cfgEdf = D.cfgEdf;
  k.flag = D.kc_flag;
  k.emax = D.kc_flag + 1;
  k.conditional = 0;
  k.shellP = D.shellP;
  k.shell_pmax = D.shell_pmax;
  k.ck_sterm = D.ck_sterm;
  k.ck_nblk = D.ck_nblk;
  k.cks_slot = D.cks_slot;
  k.cks_cfg = D.cks_cfg;
  k.cks_rep = D.cks_rep;
  k.cks_first = D.cks_first;
  k.ck_copy = D.ck_copy;
  k.ckc_dst = D.ckc_dst;
  k.ckc_src = D.ckc_src;
  k.max_copies = kcs_max_copies(P);
  k.gsum_begin = D.gsum_begin;
  k.gsum_off = D.gsum_off;
  return k;
}

// Double-float pass, then the FP64 pass (2 CTAs per SM, each looping over rows),
// whose CTAs exit at once unless a slice was not finite or no entry reached 2^-60.
template <bool MONO, bool CHUNKED, bool SHELL = false>
static lam_status launch_kcs(const Plan& P, const KcArgs& k, cudaStream_t s) {
  const size_t smem = kcs_smem(P);
  LAM_CUDA(cudaFuncSetAttribute(kc_stream<MONO, CHUNKED, true, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  LAM_CUDA(cudaFuncSetAttribute(kc_stream<MONO, CHUNKED, false, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  LAM_CUDA(cudaMemsetAsync(k.flag, 0, 2 * sizeof(int), s));
  cudaEvent_t ev = prof_begin(const_cast<Plan&>(P), s);
  kc_stream<MONO, CHUNKED, true, SHELL><<<(unsigned)P.ns, kcs_block(P), smem, s>>>(k);
  LAM_CUDA(cudaGetLastError());
  KcArgs k64 = k;
  k64.conditional = 1;
  const int64_t grid64 = std::min<int64_t>(P.ns, (int64_t)kcs_ctas_per_sm(P) * std::max(1, P.dev->n_sm));
  kc_stream<MONO, CHUNKED, false, SHELL><<<(unsigned)grid64, kcs_block(P), smem, s>>>(k64);
  LAM_CUDA(cudaGetLastError());
  prof_end(const_cast<Plan&>(P), LAM_KERNEL_COMBINE, 2, s, ev);
  return LAM_OK;
}

template <bool MONO, bool CHUNKED, bool SHELL = false>
static lam_status launch_kc(const Plan& P, const KcArgs& k, cudaStream_t s) {
  const size_t smem = kc_smem(P);
  LAM_CUDA(cudaFuncSetAttribute(kc_combine<MONO, CHUNKED, true, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  cudaEvent_t ev = prof_begin(const_cast<Plan&>(P), s);
  kc_combine<MONO, CHUNKED, true, SHELL><<<(unsigned)P.ns, kc_block(P), smem, s>>>(k);
  LAM_CUDA(cudaGetLastError());
  prof_end(const_cast<Plan&>(P), LAM_KERNEL_COMBINE, 1, s, ev);
  return LAM_OK;
}

// FP64 streaming combine. The warp-specialised form (kc_ws: one CTA per SM,
// compute threads (c, k_s, d) plus kcw_copy_threads copy threads, two slice
// buffers) when both buffers fit in shared memory; otherwise kc_stream in FP64
// (two CTAs per SM alternating their compute and copy phases).
static int kcw_copy_threads(const Plan& P) { return 896 - kcs_block(P); }
static size_t kcw_smem(const Plan& P) {
  int slots = 1;
  for (int v : P.ck_nslot) slots = std::max(slots, v);
  return (2 * (size_t)slots + 1) * kcs_stride(P) * sizeof(double) + (size_t)kcs_max_terms(P) * (32 + 8) +
         (size_t)kcs_max_copies(P) * 8 + 16 + 16;
}
static bool kcw_fits(const Plan& P) {
  return kcs_block(P) + 64 <= 896 && kcw_smem(P) <= (size_t)P.dev->smem_optin;
}
template <bool MONO, bool CHUNKED, bool SHELL = false>
static lam_status launch_kc64(const Plan& P, const KcArgs& k, cudaStream_t s) {
  if (kcw_fits(P) && !SHELL && (!CHUNKED || k.it_lo == 0)) {
    // the rows' assembled Gram blocks, read by kc_ws in one coalesced load per
    // row (once per assembly: the host-output path's slabs follow on the same
    // stream); profiled with the in-plane kernels
    cudaEvent_t eg = prof_begin(const_cast<Plan&>(P), s);
    kg_rows<<<(unsigned)P.ns, std::min(512, std::max(64, ((9 * max_len_s(P) + 31) / 32) * 32)), 0, s>>>(
        k, P.dev->Grow, P.dev->gsum_begin, P.dev->gsum_off);
    LAM_CUDA(cudaGetLastError());
    prof_end(const_cast<Plan&>(P), LAM_KERNEL_INPLANE, 1, s, eg);
  }
  cudaEvent_t ev = prof_begin(const_cast<Plan&>(P), s);
  if (kcw_fits(P)) {
    KcArgs kw = k;
    if (!SHELL) kw.G = P.dev->Grow;
    const size_t smem = kcw_smem(P);
    const int nct = kcs_block(P), block = nct + kcw_copy_threads(P);
    const int64_t grid = std::min<int64_t>(P.ns, std::max(1, P.dev->n_sm));
    // copy steps of 32 values per segment: the fewest that cover 3 len_s
    const int need = (3 * max_len_s(P) + 31) / 32;
    auto kern = need <= 3 ? kc_ws<MONO, CHUNKED, SHELL, 3> : need <= 5 ? kc_ws<MONO, CHUNKED, SHELL, 5>
                                                                        : kc_ws<MONO, CHUNKED, SHELL, 6>;
    LAM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, block, smem, s>>>(kw, nct);
  } else {
    const size_t smem = kcs_smem(P);
    LAM_CUDA(cudaFuncSetAttribute(kc_stream<MONO, CHUNKED, false, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    const int64_t grid = std::min<int64_t>(P.ns, (int64_t)kcs_ctas_per_sm(P) * std::max(1, P.dev->n_sm));
    kc_stream<MONO, CHUNKED, false, SHELL><<<(unsigned)grid, kcs_block(P), smem, s>>>(k);
  }
  LAM_CUDA(cudaGetLastError());
  prof_end(const_cast<Plan&>(P), LAM_KERNEL_COMBINE, 1, s, ev);
  return LAM_OK;
}

// Combine into `values`: streaming form when a row's slices fit, class-major
// form (FP64) otherwise; the streaming form in the plan's arithmetic.
template <bool CHUNKED>
static lam_status launch_combine(const Plan& P, const KcArgs& k, cudaStream_t s) {
  const bool df = P.arith == LAM_ARITH_DOUBLE_FLOAT;
  if (P.shell) {
    if (!use_stream(P)) return launch_kc<false, CHUNKED, true>(P, k, s);
    return df ? launch_kcs<false, CHUNKED, true>(P, k, s) : launch_kc64<false, CHUNKED, true>(P, k, s);
  }
  if (use_stream(P)) {
    if (df) return P.monoclinic ? launch_kcs<true, CHUNKED>(P, k, s) : launch_kcs<false, CHUNKED>(P, k, s);
    return P.monoclinic ? launch_kc64<true, CHUNKED>(P, k, s) : launch_kc64<false, CHUNKED>(P, k, s);
  }
  return P.monoclinic ? launch_kc<true, CHUNKED>(P, k, s) : launch_kc<false, CHUNKED>(P, k, s);
}

// K-a: the configuration-free in-plane Gram blocks of every element, into EG.
static lam_status inplane_gram(Plan& P, cudaStream_t s) {
  Device& D = *P.dev;
  KaLocalArgs ka{};
  ka.ip = inplane_args(P);
  ka.nel = P.u.nel * P.v.nel;
  ka.EG = D.EG;
  const size_t smem = ka_smem(P);
  const bool df = P.arith == LAM_ARITH_DOUBLE_FLOAT;
  LAM_CUDA(cudaFuncSetAttribute(df ? ka_local : ka_local64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaEvent_t ev = prof_begin(P, s);
  if (df)
    ka_local<<<ka.nel, ka_block(P), smem, s>>>(ka);
  else
    ka_local64<<<ka.nel, ka_block(P), smem, s>>>(ka);
  LAM_CUDA(cudaGetLastError());
  prof_end(P, LAM_KERNEL_INPLANE, 1, s, ev);
  return LAM_OK;
}

// General extrusion: the 6 x 6 element Gram blocks (ka_shell), then P of
// every configuration per in-plane pair (kp_shell), into D.shellP.
static KpShellArgs kp_shell_args(const Plan& P) {
  const Device& D = *P.dev;
  KpShellArgs kp{};
  kp.nx = P.u.n;
  kp.nel_u = P.u.nel;
  kp.nlx = P.u.p + 1;
  kp.nls = ka_nls(P);
  kp.npl = ka_npl(P);
  kp.ncfg = (int)P.cfg_mat.size();
  kp.nnz_s = P.nnz_s;
  kp.LSb = D.LSb;
  kp.lenX = D.lenX;
  kp.lenY = D.lenY;
  kp.loX = D.loX;
  kp.loY = D.loY;
  kp.eloX = D.eloX;
  kp.ehiX = D.ehiX;
  kp.eloY = D.eloY;
  kp.ehiY = D.ehiY;
  kp.firstU = D.firstU;
  kp.firstV = D.firstV;
  kp.EG = D.shellEG;
  return kp;
}

// K-a of a general extrusion: the 6 x 6 element Gram blocks into D.shellEG.
static lam_status shell_element_gram(Plan& P, cudaStream_t s) {
  Device& D = *P.dev;
  const int nel = P.u.nel * P.v.nel, npl = ka_npl(P);
  if (!D.shellEG && alloc_dev(D.allocs, &D.shellEG, (size_t)nel * 36 * npl) != LAM_OK) return LAM_ERR_OOM;
  KaShellArgs ka{};
  ka.ip = inplane_args(P);
  ka.EG = D.shellEG;
  if (P.arith == LAM_ARITH_DOUBLE_FLOAT) {
    const size_t smem = ka_shell_smem(P);
    LAM_CUDA(cudaFuncSetAttribute(ka_shell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ka_shell<<<(unsigned)nel, 256, smem, s>>>(ka);
  } else {
    const size_t smem = ka_shell64_smem(P);
    LAM_CUDA(cudaFuncSetAttribute(ka_shell64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ka_shell64<<<(unsigned)nel, 256, smem, s>>>(ka);
  }
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

static lam_status shell_operators(Plan& P, cudaStream_t s, bool full) {
  Device& D = *P.dev;
  const int ncfg = (int)P.cfg_mat.size();
  if (!D.shell_pmax) {
    double* pm = nullptr;
    if (alloc_dev(D.allocs, &pm, 4) != LAM_OK) return LAM_ERR_OOM;
    D.shell_pmax = reinterpret_cast<unsigned long long*>(pm);
  }
  const size_t need = (size_t)ncfg * P.nnz_s * 36;
  if (D.shellP_elems < need) {
    if (D.shellP) cudaFree(D.shellP);
    D.shellP = nullptr;
    D.shellP_elems = 0;
    cudaError_t e = device_alloc(reinterpret_cast<void**>(&D.shellP), need * sizeof(double));
    if (e != cudaSuccess) {
      set_error("cudaMalloc(P of the general extrusion, %zu doubles) failed: %s", need, cudaGetErrorString(e));
      return LAM_ERR_OOM;
    }
    D.shellP_elems = need;
  }
  cudaEvent_t ev = prof_begin(P, s);
  lam_status st = shell_element_gram(P, s);
  if (st != LAM_OK) return st;
  KpShellArgs kp = kp_shell_args(P);
  kp.Edf = D.shell_Edf;
  kp.kE = D.shell_kE;
  kp.P = D.shellP;
  kp.pmax = D.shell_pmax;
  kp.full = full ? 1 : 0;
  LAM_CUDA(cudaMemsetAsync(D.shell_pmax, 0, 4 * sizeof(unsigned long long), s));
  const bool smem_e = ncfg <= kKpShellSmemCfg;
  // threads for the pairs j_s >= i_s of an interior row (about half); rows with more loop
  const int block_p = std::max(64, ((4 * (max_len_s(P) / 2 + 1) + 31) / 32) * 32);
  if (P.arith == LAM_ARITH_DOUBLE_FLOAT) {
    const size_t smem_p = smem_e ? (size_t)ncfg * 81 * sizeof(float2) : 0;
    auto kern = smem_e ? (P.monoclinic ? kp_shell<true, true> : kp_shell<true, false>)
                       : (P.monoclinic ? kp_shell<false, true> : kp_shell<false, false>);
    LAM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
    kern<<<(unsigned)P.ns, block_p, smem_p, s>>>(kp);
  } else {
    const size_t smem_p = smem_e ? (size_t)ncfg * 81 * sizeof(double) : 0;
    auto kern = smem_e ? (P.monoclinic ? kp_shell64<true, true> : kp_shell64<true, false>)
                       : (P.monoclinic ? kp_shell64<false, true> : kp_shell64<false, false>);
    LAM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
    kern<<<(unsigned)P.ns, block_p, smem_p, s>>>(kp, D.cfgE);
  }
  LAM_CUDA(cudaGetLastError());
  prof_end(P, LAM_KERNEL_INPLANE, 2, s, ev);
  return LAM_OK;
}

// K-b then K-a: leaves Q and the element Gram blocks in the plan's workspace.
static lam_status split_integrals(Plan& P, cudaStream_t s) {
  Device& D = *P.dev;
  KbArgs kb{};
  kb.npairs = P.nnz_t;
  kb.ncfg = (int)P.cfg_mat.size();
  kb.nqt = P.nqt;
  kb.q1 = P.t.p + 1;
  kb.tp_row = D.tp_row;
  kb.tp_col = D.tp_col;
  kb.tp_e0 = D.tp_e0;
  kb.tp_e1 = D.tp_e1;
  kb.firstT = D.firstT;
  kb.piece_begin = D.piece_begin;
  kb.piece_cfg = D.piece_cfg;
  kb.tabT = D.tabT;
  kb.wT = D.wT;
  kb.q = D.q;
  kb.qdf = D.qdf;
  // Eq. Q depends on the plies only: computed on the first call and after every
  // lam_plan_update (which replaces the configuration tables), kept otherwise.
  // K-b (a few microseconds) runs beside K-a: forked after the work already on
  // the caller's stream, joined before the combine.
  const bool run_kb = !D.q_valid;
  if (run_kb) {
    if (!D.kb_stream) {
      LAM_CUDA(cudaStreamCreateWithFlags(&D.kb_stream, cudaStreamNonBlocking));
      LAM_CUDA(cudaEventCreateWithFlags(&D.kb_fork, cudaEventDisableTiming));
      LAM_CUDA(cudaEventCreateWithFlags(&D.kb_join, cudaEventDisableTiming));
    }
    LAM_CUDA(cudaEventRecord(D.kb_fork, s));
    LAM_CUDA(cudaStreamWaitEvent(D.kb_stream, D.kb_fork, 0));
    cudaEvent_t ev = prof_begin(P, D.kb_stream);
    kb_thickness<<<(unsigned)((P.nnz_t + 127) / 128), 128, 0, D.kb_stream>>>(kb);
    LAM_CUDA(cudaGetLastError());
    prof_end(P, LAM_KERNEL_THICKNESS, 1, D.kb_stream, ev);
    LAM_CUDA(cudaEventRecord(D.kb_join, D.kb_stream));
    D.q_valid = true;
  }
  const lam_status st = P.shell ? shell_operators(P, s, false) : inplane_gram(P, s);
  if (run_kb) LAM_CUDA(cudaStreamWaitEvent(s, D.kb_join, 0));
  return st;
}

// ---------------------------------------------------------------------------
// Adjoint (lam_adjoint). K is linear in every ply's D_l; with the split of
// Section 3 the coefficient of the stored entry (i_t i_s c, j_t j_s d) in
// D_l[V(c,a)][V(d,b)] is G_ab^{i_s j_s} Q_{l,ab}^{i_t j_t} (Eq. Km_2, with
// Eq. P and Eq. Q restricted to ply l), so
//   S_l[cd][ab] = sum over stored entries of gbar * G_ab * Q_{l,ab}.
// adj_ply evaluates it thickness first: CTA (chunk of in-plane rows, ply l),
// thread (c, k_s, d). Per row, z_type = sum over the ply's thickness pairs of
// gbar * Q_type (types T T, T T', T' T, T' T'), then S[ab] += z_type(ab) *
// G_ab(i_s, k_s); at the end the CTA sums S over k_s (fixed order) into one
// partial per (ply, chunk). Q and G enter divided by powers of two (exact), so
// the double-float arithmetic stays far from float overflow; adj_reduce
// multiplies the scales back, folds the 81 (cd, ab) sums onto the 36 entries of
// dL/dD_l and applies the chain rule through Eq. D.
// ---------------------------------------------------------------------------
constexpr int kAdjRows = 16;        // in-plane rows per CTA
constexpr int kAdjMaxTerms = 1024;  // thickness pairs meeting one ply
constexpr int kAdjBatch = 8;        // cotangent loads issued together
// The double-float pass is kept only if the largest cotangent magnitude is at
// least 2^(kAdjMinExp - 1023); below that (a cotangent of tiny entries only)
// the FP64 pass recomputes everything, as it does for non-finite partials.
constexpr int kAdjMinExp = 1023 - 60;
// ... and likewise when an entry (low-rank: a product of entries) reaches 2^128.
constexpr int kAdjMaxExp = 1150;

struct AdjGatherArgs {
  int nx, nel_u, nlx, nls, npl;
  const int64_t* LSb;
  const int *lenX, *lenY, *loX, *loY, *eloX, *ehiX, *eloY, *ehiY, *firstU, *firstV;
  const double* EG;
  double* G;                   // nnz_s x 9
  unsigned long long* gmax;    // 9 maxima of |G_ab| as bit patterns
};

// Assembled in-plane Gram blocks G_ab(i_s, k_s) (the sum over the shared
// elements, in a fixed element order) and the maxima of |G_ab|.
__global__ void __launch_bounds__(1024) adj_gather(AdjGatherArgs a) {
  __shared__ unsigned long long smax[9];
  if (threadIdx.x < 9) smax[threadIdx.x] = 0ull;
  __syncthreads();
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  for (int item = threadIdx.x; item < 9 * ls; item += blockDim.x) {
    const int ks = item / 9, ab = item % 9;
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
    const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
    const int ba = (ab % 3) * 3 + ab / 3;
    double acc = 0.0;
    for (int ey = ey0; ey <= ey1; ++ey) {
      const int fy = a.firstV[ey];
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        const size_t ep = ((size_t)ey * a.nel_u + ex) * a.npl;
        if (li <= lj)
          acc += a.EG[(ep + upper_pair(li, lj, a.nls)) * 9 + ab];
        else
          acc += a.EG[(ep + upper_pair(lj, li, a.nls)) * 9 + ba];
      }
    }
    a.G[(ls0 + ks) * 9 + ab] = acc;
    atomicMax(&smax[ab], (unsigned long long)__double_as_longlong(fabs(acc)));
  }
  __syncthreads();
  if (threadIdx.x < 9) atomicMax(&a.gmax[threadIdx.x], smax[threadIdx.x]);
}

// G_ab divided by a power of two at least max |G_ab| (exact), and its float
// pairs. The 9 scales go to gscale.
__global__ void adj_split(int64_t n9, double* __restrict__ G, float2* __restrict__ Gdf,
                          const unsigned long long* __restrict__ gmax, double* __restrict__ gscale) {
  __shared__ double inv[9];
  if (threadIdx.x < 9) {
    const double m = __longlong_as_double((long long)gmax[threadIdx.x]);
    double sc = 1.0;
    if (m > 0.0 && m <= 1.7976931348623157e308) {
      int e = 0;
      frexp(m, &e);
      sc = ldexp(1.0, e);
    }
    inv[threadIdx.x] = 1.0 / sc;
    if (blockIdx.x == 0) gscale[threadIdx.x] = sc;
  }
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n9; k += (int64_t)gridDim.x * blockDim.x) {
    const double g = G[k] * inv[k % 9];
    G[k] = g;
    float hi, lo;
    split_df(g, hi, lo);
    Gdf[k] = make_float2(hi, lo);
  }
}

struct AdjArgs {
  int64_t ns, n_dof;
  int nx, lsp, nchunks, mt;
  const int64_t* LSb;
  const int *lenX, *lenY, *loX, *loY;
  const int *term_begin, *term_pair;
  const double* term_q;     // [term][4], scaled
  const float* term_qdf;    // [term][8]: hi[4], lo[4]
  const int64_t* tp_A;
  const int *tp_lt, *tp_k, *tp_row, *tp_col;
  const double* gbar;       // CSR cotangent
  const double *u, *v;      // low-rank cotangent, rank x n_dof each
  int rank;
  const double* G;          // scaled G, nnz_s x 9
  const float2* Gdf;        // its float pairs
  double* partial;          // n_plies x nchunks x 81
  int* flag;                // set by the double-float pass on a non-finite partial
  int* emax;                // largest biased exponent of the cotangent seen by that pass
  int conditional;          // run only if the double-float result is not kept
  // general extrusion (FP64 pass): the 6 x 6 Gram blocks G_(alpha a)(beta b) of
  // every in-plane pair, unscaled, and the scales of the four Q types
  const double* G36;        // nnz_s x 36, [blk * 9 + ab]
  double qs[4];
  // ... and for the double-float pass: qs[blk] G_(blk)(ab) / gscale[ab] as float pairs
  const float2* G36df;
};

// SHELL: a general extrusion, whose entry (c, d) of K couples every (a, b) of
// D_l through all four thickness types: S[ab] += sum_type z_type G_(type)(ab)
// (FP64 only).
template <bool LOWRANK, bool DF, bool SHELL = false>
__global__ void __launch_bounds__(1024) adj_ply(AdjArgs a) {
  static_assert(!(SHELL && DF), "general extrusions take the FP64 pass");
  if (a.conditional && *a.flag == 0 && *a.emax >= kAdjMinExp && *a.emax <= kAdjMaxExp) return;
  extern __shared__ double sm[];
  const int l = blockIdx.y, chunk = blockIdx.x;
  const int t0 = a.term_begin[l], nterm = a.term_begin[l + 1] - t0;
  const int nthr = blockDim.x, tid = threadIdx.x;
  int64_t* sA = reinterpret_cast<int64_t*>(sm);           // CSR slab start of the pair's thickness row
  double* sQ = sm + a.mt;                                  // Q (4 doubles, or 8 floats: hi[4] lo[4])
  int* sI = reinterpret_cast<int*>(sQ + 4 * (size_t)a.mt);  // len_t, k_t, i_t, j_t
  double* red = reinterpret_cast<double*>(sI + 4 * (size_t)a.mt);  // 9 x nthr
  for (int k = tid; k < nterm; k += nthr) {
    const int pr = a.term_pair[t0 + k];
    sA[k] = a.tp_A[pr];
    sI[4 * k + 0] = a.tp_lt[pr];
    sI[4 * k + 1] = a.tp_k[pr];
    sI[4 * k + 2] = a.tp_row[pr];
    sI[4 * k + 3] = a.tp_col[pr];
    if (DF) {
      float* q = reinterpret_cast<float*>(sQ + 4 * (size_t)k);
#pragma unroll
      for (int j = 0; j < 8; ++j) q[j] = a.term_qdf[(size_t)(t0 + k) * 8 + j];
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) sQ[4 * (size_t)k + j] = a.term_q[(size_t)(t0 + k) * 4 + j];
    }
  }
  __syncthreads();
  const int lsp3 = 3 * a.lsp;
  const bool valid = tid < 9 * a.lsp;
  const int c = valid ? tid / lsp3 : 0, rem = valid ? tid % lsp3 : 0;
  const int ks = rem / 3, d = rem % 3;
  float Sh[9], Sl[9];
  double S[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Sh[k] = Sl[k] = 0.0f;
    S[k] = 0.0;
  }
  int emax = 0;
  const int64_t r0 = (int64_t)chunk * kAdjRows;
  for (int r = 0; r < kAdjRows; ++r) {
    const int64_t is = r0 + r;
    if (is >= a.ns) break;
    const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
    const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
    if (!valid || ks >= ls) continue;
    const int64_t ls0 = a.LSb[is];
    const int64_t rowbase = 9 * ls0 + 3 * (int64_t)c * ls;
    const int off = 3 * ks + d, seg = 3 * ls;
    int64_t jbase = 0;
    if (LOWRANK) {
      const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
      jbase = (int64_t)jy * a.nx + jx;
    }
    float zh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, zl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    for (int tb = 0; tb < nterm; tb += kAdjBatch) {
      double gv[kAdjBatch];
      if (!LOWRANK) {
#pragma unroll
        for (int j = 0; j < kAdjBatch; ++j) {
          const int t = tb + j;
          gv[j] = (t < nterm) ? a.gbar[sA[t] + sI[4 * t] * rowbase + (int64_t)sI[4 * t + 1] * seg + off] : 0.0;
        }
      }
#pragma unroll
      for (int j = 0; j < kAdjBatch; ++j) {
        const int t = tb + j;
        if (t >= nterm) break;
        if (DF) {
          float gh = 0.0f, gl = 0.0f;
          if (LOWRANK) {
            const int64_t iu = 3 * ((int64_t)sI[4 * t + 2] * a.ns + is) + c;
            const int64_t iv = 3 * ((int64_t)sI[4 * t + 3] * a.ns + jbase) + d;
            for (int q = 0; q < a.rank; ++q) {
              float uh, ul, vh, vl, p, e;
              const int eu = split_df(a.u[(size_t)q * a.n_dof + iu], uh, ul);
              const int ev = split_df(a.v[(size_t)q * a.n_dof + iv], vh, vl);
              if (eu > 0 && ev > 0) emax = max(emax, eu + ev - 1023);
              df_mul(uh, ul, vh, vl, p, e);
              df_add(p, e, gh, gl);
            }
          } else {
            emax = max(emax, split_df(gv[j], gh, gl));
          }
          const float* q = reinterpret_cast<const float*>(sQ + 4 * (size_t)t);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float p, e;
            df_mul(gh, gl, q[k], q[4 + k], p, e);
            df_add(p, e, zh[k], zl[k]);
          }
        } else {
          double g = LOWRANK ? 0.0 : gv[j];
          if (LOWRANK) {
            const int64_t iu = 3 * ((int64_t)sI[4 * t + 2] * a.ns + is) + c;
            const int64_t iv = 3 * ((int64_t)sI[4 * t + 3] * a.ns + jbase) + d;
            g = 0.0;
            for (int q = 0; q < a.rank; ++q) g += a.u[(size_t)q * a.n_dof + iu] * a.v[(size_t)q * a.n_dof + iv];
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) z[k] += g * sQ[4 * (size_t)t + k];
        }
      }
    }
    // S[ab] += z_type(ab) * G_ab, type(ab) = 2 [a is z] + [b is z]
    const int64_t gi = (ls0 + ks) * 9;
    if (DF) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // renormalise the pairs
        const float hsum = __fadd_rn(zh[k], zl[k]);
        zl[k] = __fsub_rn(zl[k], __fsub_rn(hsum, zh[k]));
        zh[k] = hsum;
      }
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int ty = 2 * (ab / 3 == 2) + (ab % 3 == 2);
        const float2 gq = a.Gdf[gi + ab];
        float p, e;
        df_mul(zh[ty], zl[ty], gq.x, gq.y, p, e);
        df_add(p, e, Sh[ab], Sl[ab]);
      }
    } else if (SHELL) {
      const double* g36 = a.G36 + (ls0 + ks) * 36;
      const double z0 = z[0] * a.qs[0], z1 = z[1] * a.qs[1], z2 = z[2] * a.qs[2], z3 = z[3] * a.qs[3];
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) S[ab] += z0 * g36[ab] + z1 * g36[9 + ab] + z2 * g36[18 + ab] + z3 * g36[27 + ab];
    } else {
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int ty = 2 * (ab / 3 == 2) + (ab % 3 == 2);
        S[ab] += z[ty] * a.G[gi + ab];
      }
    }
  }
  if (DF) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((tid & 31) == 0) atomicMax(a.emax, emax);
  }
  __syncthreads();
#pragma unroll
  for (int ab = 0; ab < 9; ++ab)
    red[(size_t)ab * nthr + tid] = valid ? (DF ? (double)Sh[ab] + (double)Sl[ab] : S[ab]) : 0.0;
  __syncthreads();
  if (tid < 81) {
    const int cd = tid / 9, ab = tid % 9, cc = cd / 3, dd = cd % 3;
    double acc = 0.0;
    for (int k = 0; k < a.lsp; ++k) acc += red[(size_t)ab * nthr + cc * lsp3 + 3 * k + dd];
    a.partial[((size_t)l * a.nchunks + chunk) * 81 + tid] = acc;
    if (DF && !isfinite(acc)) atomicOr(a.flag, 1);
  }
}

// Double-float pass for a CSR cotangent (the common case), leaner than the
// generic kernel: the CTA first tabulates, in shared memory, the CSR offset of
// every (row of its chunk, c, thickness pair of its ply) -- 32-bit when
// nnz < 2^31 -- so a thread's load is one shared read and one add; all of a
// row's cotangent loads of one batch are issued before any arithmetic; the four
// Q types of a term come from shared memory as two float4. Used when a ply
// meets at most kAdjFastTerms thickness pairs.
constexpr int kAdjRowTerms = 9;
constexpr int kAdjFastTerms = 32;

template <typename Idx, bool SHELL = false>
__global__ void __launch_bounds__(1024) adj_ply_df(AdjArgs a) {
  extern __shared__ double sm[];
  const int l = blockIdx.y, chunk = blockIdx.x;
  const int t0 = a.term_begin[l], nterm = a.term_begin[l + 1] - t0;
  const int nthr = blockDim.x, tid = threadIdx.x;
  float4* sQh = reinterpret_cast<float4*>(sm);                  // kAdjFastTerms
  float4* sQl = sQh + kAdjFastTerms;                             // kAdjFastTerms
  double* sQ3 = reinterpret_cast<double*>(sQl + kAdjFastTerms);  // kAdjFastTerms: the T' T' type in FP64
  double* red = sQ3 + kAdjFastTerms;                             // 9 x nthr
  Idx* sBase = reinterpret_cast<Idx*>(red + (size_t)9 * nthr);   // kAdjRows x 3 x kAdjFastTerms
  int* sLs = reinterpret_cast<int*>(sBase + kAdjRows * 3 * kAdjFastTerms);  // kAdjRows
  int* sLs0 = sLs + kAdjRows;                                    // kAdjRows (in-plane pair offset of the row)
  const int64_t r0 = (int64_t)chunk * kAdjRows;
  const int nrows = (int)min((int64_t)kAdjRows, a.ns - r0);
  for (int k = tid; k < nterm; k += nthr) {
    const float* q = a.term_qdf + (size_t)(t0 + k) * 8;
    sQh[k] = make_float4(q[0], q[1], q[2], q[3]);
    sQl[k] = make_float4(q[4], q[5], q[6], q[7]);
    sQ3[k] = a.term_q[(size_t)(t0 + k) * 4 + 3];
  }
  if (tid < nrows) {
    const int is = (int)(r0 + tid);
    sLs[tid] = a.lenX[is % a.nx] * a.lenY[is / a.nx];
    sLs0[tid] = (int)a.LSb[is];
  }
  __syncthreads();
  for (int k = tid; k < nrows * 3 * nterm; k += nthr) {
    const int r = k / (3 * nterm), c3 = (k / nterm) % 3, t = k % nterm;
    const int pr = a.term_pair[t0 + t];
    const int64_t ls = sLs[r];
    sBase[(r * 3 + c3) * kAdjFastTerms + t] =
        (Idx)(a.tp_A[pr] + (int64_t)a.tp_lt[pr] * (9 * (int64_t)sLs0[r] + 3 * c3 * ls) + (int64_t)a.tp_k[pr] * 3 * ls);
  }
  __syncthreads();
  const int lsp3 = 3 * a.lsp;
  const bool valid = tid < 9 * a.lsp;
  const int c = valid ? tid / lsp3 : 0, rem = valid ? tid % lsp3 : 0;
  const int ks = rem / 3, d = rem % 3;
  float Sh[9], Sl[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Sh[k] = Sl[k] = 0.0f;
  int emax = 0;
  for (int r = 0; r < nrows; ++r) {
    const int ls = sLs[r];
    if (!valid || ks >= ls) continue;
    const Idx* bp = sBase + (r * 3 + c) * kAdjFastTerms;
    const Idx off = (Idx)(3 * ks + d);
    // types T T, T T', T' T in double-float on the FP32 pipes; T' T' in FP64 on
    // the otherwise idle FP64 pipe, which runs alongside
    float zh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, zl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    double z3 = 0.0;
    for (int tb = 0; tb < nterm; tb += kAdjRowTerms) {
      double v[kAdjRowTerms];
#pragma unroll
      for (int j = 0; j < kAdjRowTerms; ++j) v[j] = (tb + j < nterm) ? a.gbar[bp[tb + j] + off] : 0.0;
#pragma unroll
      for (int j = 0; j < kAdjRowTerms; ++j) {
        const int t = tb + j;
        if (t < nterm) {
          float gh, gl;
          emax = max(emax, split_df_fast(v[j], gh, gl));
          const float4 qh = sQh[t], ql = sQl[t];
          float p, e;
          df_mul(gh, gl, qh.x, ql.x, p, e);
          df_add(p, e, zh[0], zl[0]);
          df_mul(gh, gl, qh.y, ql.y, p, e);
          df_add(p, e, zh[1], zl[1]);
          df_mul(gh, gl, qh.z, ql.z, p, e);
          df_add(p, e, zh[2], zl[2]);
          z3 = __fma_rn(v[j], sQ3[t], z3);
        }
      }
    }
    split_df(z3, zh[3], zl[3]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // renormalise the pairs
      const float hsum = __fadd_rn(zh[k], zl[k]);
      zl[k] = __fsub_rn(zl[k], __fsub_rn(hsum, zh[k]));
      zh[k] = hsum;
    }
    if (SHELL) {  // S[ab] += sum_type z_type G_(type)(ab), all four types
      const float2* gp = a.G36df + ((int64_t)sLs0[r] + ks) * 36;
#pragma unroll
      for (int ab = 0; ab < 9; ++ab)
#pragma unroll
        for (int ty = 0; ty < 4; ++ty) {
          const float2 gq = gp[ty * 9 + ab];
          float p, e;
          df_mul(zh[ty], zl[ty], gq.x, gq.y, p, e);
          df_add(p, e, Sh[ab], Sl[ab]);
        }
    } else {
      const float2* gp = a.Gdf + ((int64_t)sLs0[r] + ks) * 9;
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int ty = 2 * (ab / 3 == 2) + (ab % 3 == 2);
        const float2 gq = gp[ab];
        float p, e;
        df_mul(zh[ty], zl[ty], gq.x, gq.y, p, e);
        df_add(p, e, Sh[ab], Sl[ab]);
      }
    }
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  if ((tid & 31) == 0) atomicMax(a.emax, emax);
  __syncthreads();
#pragma unroll
  for (int ab = 0; ab < 9; ++ab) red[(size_t)ab * nthr + tid] = valid ? (double)Sh[ab] + (double)Sl[ab] : 0.0;
  __syncthreads();
  if (tid < 81) {
    const int cd = tid / 9, ab = tid % 9, cc = cd / 3, dd = cd % 3;
    double acc = 0.0;
    for (int k = 0; k < a.lsp; ++k) acc += red[(size_t)ab * nthr + cc * lsp3 + 3 * k + dd];
    a.partial[((size_t)l * a.nchunks + chunk) * 81 + tid] = acc;
    if (!isfinite(acc)) atomicOr(a.flag, 1);
  }
}

static size_t adj_df_smem(int nthr, size_t idx_bytes) {
  return (size_t)kAdjFastTerms * 40 + (size_t)9 * nthr * sizeof(double) + (size_t)kAdjRows * 3 * kAdjFastTerms * idx_bytes +
         2 * kAdjRows * sizeof(int);
}

// ---------------------------------------------------------------------------
// Low-rank cotangent (L = sum_q u_q^T K v_q), factorised: with scaled G,
//   W_q(j_t, i_s)[ab][d] = sum_{k_s} G_ab(i_s, k_s) v_q(j_t, j_s(k_s), d),
//   X(i_t, j_t)[c][d][ab] = sum_q sum_{i_s} u_q(i_t, i_s, c) W_q(j_t, i_s)[ab][d],
//   S_l[cd][ab] = sum over the ply's thickness pairs of Q_{l,type(ab)} X,
// in FP64 (about 9 FMA per in-plane pair, thickness function and rank, against
// 9 per stored entry for the general cotangent).
// ---------------------------------------------------------------------------
struct AdjLrArgs {
  int64_t ns, nt, n_dof;
  int nx;
  const int64_t* LSb;
  const int *lenX, *lenY, *loX, *loY;
  const double* G;
  const double* u;  // rank q's vectors (offset applied by the host)
  const double* v;
  double* W;
  double* X;
  int64_t npairs;
  const int *tp_row, *tp_col;
  int accumulate;   // add to X (ranks after the first)
};

__global__ void adj_lr_w(AdjLrArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.nt * a.ns * 27) return;
  const int k = (int)(t % 27);
  const int64_t r = t / 27, is = r % a.ns, jt = r / a.ns;
  const int ab = k / 3, d = k % 3;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  double acc = 0.0;
  for (int ks = 0; ks < ls; ++ks) {
    const int64_t js = (int64_t)(a.loY[iy] + ks / lx) * a.nx + a.loX[ix] + ks % lx;
    acc += a.G[(ls0 + ks) * 9 + ab] * a.v[3 * (jt * a.ns + js) + d];
  }
  a.W[t] = acc;
}

// One CTA per thickness pair, 3 x 81 threads: each sums a third of the
// in-plane functions, then the thirds are added in a fixed order.
__global__ void __launch_bounds__(256) adj_lr_x(AdjLrArgs a) {
  __shared__ double part[3][81];
  const int64_t pr = blockIdx.x;
  const int it = a.tp_row[pr], jt = a.tp_col[pr];
  const int t = threadIdx.x;
  if (t < 243) {
    const int o = t % 81, q = t / 81;
    const int c = o / 27, dab = o % 27;  // o = (c * 3 + d) * 9 + ab
    const int d = (o / 9) % 3, ab = o % 9;
    (void)dab;
    double acc = 0.0;
    for (int64_t is = q; is < a.ns; is += 3)
      acc += a.u[3 * ((int64_t)it * a.ns + is) + c] * a.W[((int64_t)jt * a.ns + is) * 27 + ab * 3 + d];
    part[q][o] = acc;
  }
  __syncthreads();
  if (t < 81) {
    const double v = (part[0][t] + part[1][t]) + part[2][t];
    a.X[pr * 81 + t] = a.accumulate ? a.X[pr * 81 + t] + v : v;
  }
}

// Per ply: S_l[cd][ab] = sum over its terms of Q_{type(ab)} X(pair), written as
// the ply's single partial for adj_reduce.
__global__ void adj_lr_ply(const int* __restrict__ term_begin, const int* __restrict__ term_pair,
                           const double* __restrict__ term_q, const double* __restrict__ X, double* __restrict__ partial) {
  const int l = blockIdx.x, t = threadIdx.x;
  if (t >= 81) return;
  const int ab = t % 9;
  const int ty = 2 * (ab / 3 == 2) + (ab % 3 == 2);
  double acc = 0.0;
  for (int k = term_begin[l]; k < term_begin[l + 1]; ++k) acc += term_q[(size_t)k * 4 + ty] * X[(size_t)term_pair[k] * 81 + t];
  partial[(size_t)l * 81 + t] = acc;
}

struct AdjReduceArgs {
  int nchunks;
  double qscale[4];
  const double* gscale;
  const double* partial;
  const double *ply_M, *ply_dM, *mat_C;
  const int* ply_mat;
  double *dD, *dtheta, *plyC;
};

// One CTA per ply: the 81 sums (scales restored), dL/dD_l, dL/dtheta_l and
// the ply's share of dL/dC (21 constants).
__global__ void __launch_bounds__(384) adj_reduce(AdjReduceArgs a) {
  __shared__ double S[81], dD[36], pr[36], T[36], part[4][81];
  const int l = blockIdx.x, t = threadIdx.x;
  if (t < 4 * 81) {  // four threads per sum, then a fixed-order combination
    const int k = t % 81, q = t / 81;
    double acc = 0.0;
    for (int ch = q; ch < a.nchunks; ch += 4) acc += a.partial[((size_t)l * a.nchunks + ch) * 81 + k];
    part[q][k] = acc;
  }
  __syncthreads();
  if (t < 81) {
    const int ab = t % 9;
    const int ty = 2 * (ab / 3 == 2) + (ab % 3 == 2);
    S[t] = (((part[0][t] + part[1][t]) + part[2][t]) + part[3][t]) * a.qscale[ty] * a.gscale[ab];
  }
  __syncthreads();
  // Voigt index of the symmetric pair (i, j): 11, 22, 33, 12, 13, 23
  const int V[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  if (t < 36) {
    const int I = t / 6, J = t % 6;
    double acc = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int x = 0; x < 3; ++x) {
        if (V[c][x] != I) continue;
        for (int d = 0; d < 3; ++d)
          for (int y = 0; y < 3; ++y)
            if (V[d][y] == J) acc += S[(c * 3 + d) * 9 + x * 3 + y];
      }
    dD[t] = acc;
    if (a.dD) a.dD[(size_t)l * 36 + t] = acc;
  }
  __syncthreads();
  const double* M = a.ply_M + (size_t)l * 36;
  const double* dM = a.ply_dM + (size_t)l * 36;
  const double* C = a.mat_C + (size_t)a.ply_mat[l] * 36;
  if (t < 36) {
    const int I = t / 6, J = t % 6;
    double x = 0.0, y = 0.0;
    for (int K = 0; K < 6; ++K)
      for (int L = 0; L < 6; ++L) {
        x += (dM[I * 6 + K] * M[J * 6 + L] + M[I * 6 + K] * dM[J * 6 + L]) * C[K * 6 + L];
        y += M[K * 6 + I] * dD[K * 6 + L] * M[L * 6 + J];
      }
    pr[t] = dD[t] * x;
    T[t] = y;
  }
  __syncthreads();
  if (t == 0 && a.dtheta) {
    double acc = 0.0;
    for (int k = 0; k < 36; ++k) acc += pr[k];
    a.dtheta[l] = acc;
  }
  if (t < 21) {
    int p = 0, r = t;
    while (r >= 6 - p) {
      r -= 6 - p;
      ++p;
    }
    const int q = p + r;
    a.plyC[(size_t)l * 21 + t] = (p == q) ? T[p * 6 + q] : T[p * 6 + q] + T[q * 6 + p];
  }
}

// dL/dC_m = sum over the plies of material m, in ply order.
__global__ void adj_material(int nply, int nmat, const int* __restrict__ ply_mat, const double* __restrict__ plyC,
                             double* __restrict__ dC) {
  for (int k = threadIdx.x; k < nmat * 21; k += blockDim.x) {
    const int m = k / 21, j = k % 21;
    double acc = 0.0;
    for (int l = 0; l < nply; ++l)
      if (ply_mat[l] == m) acc += plyC[(size_t)l * 21 + j];
    dC[k] = acc;
  }
}

static int adj_nchunks(const Plan& P) { return (int)((P.ns + kAdjRows - 1) / kAdjRows); }
static int adj_block(const Plan& P) { return std::max(96, ((9 * max_len_s(P) + 31) / 32) * 32); }
static size_t adj_smem(const Plan& P) {
  // generic kernel: per term 8 (offset) + 32 (Q) + 16 (indices); fast kernel: 32 + 8 + 8 and 16 bytes of
  // alignment slack. The larger of the two, then the reduction buffer.
  return (size_t)P.adj_max_terms * (8 + 32 + 16) + 16 + (size_t)9 * adj_block(P) * sizeof(double);
}

static lam_status ensure_adjoint_alloc(Plan& P);
// The adjoint's workspace; a failed allocation releases what this call allocated.
static lam_status ensure_adjoint(Plan& P) {
  Device& D = *P.dev;
  if (D.adj_ready) return LAM_OK;
  const size_t mark = D.allocs.size();
  const lam_status st = ensure_adjoint_alloc(P);
  if (st != LAM_OK) {
    for (size_t k = mark; k < D.allocs.size(); ++k) cudaFree(D.allocs[k]);
    D.allocs.resize(mark);
  }
  return st;
}
static lam_status ensure_adjoint_alloc(Plan& P) {
  Device& D = *P.dev;
  lam_status st;
  auto& L = D.allocs;
  if ((st = upload(P, L, &D.adj_begin, P.adj_begin)) != LAM_OK) return st;
  if ((st = upload(P, L, &D.adj_pair, P.adj_pair)) != LAM_OK) return st;
  if ((st = upload(P, L, &D.adj_q, P.adj_q)) != LAM_OK) return st;
  if ((st = upload(P, L, &D.adj_qdf, P.adj_qdf)) != LAM_OK) return st;
  double* p = nullptr;
  if ((st = alloc_dev(L, &D.adj_G, (size_t)9 * P.nnz_s)) != LAM_OK) return st;
  if ((st = alloc_dev(L, &p, (size_t)9 * P.nnz_s)) != LAM_OK) return st;
  D.adj_Gdf = reinterpret_cast<float2*>(p);
  if ((st = alloc_dev(L, &p, 18)) != LAM_OK) return st;
  D.adj_gmax = reinterpret_cast<unsigned long long*>(p);
  if ((st = alloc_dev(L, &D.adj_partial, (size_t)P.plies.size() * adj_nchunks(P) * 81)) != LAM_OK) return st;
  if ((st = alloc_dev(L, &D.adj_plyC, (size_t)P.plies.size() * 21)) != LAM_OK) return st;
  if ((st = alloc_dev(L, &D.adj_W, (size_t)P.nt * P.ns * 27)) != LAM_OK) return st;
  if ((st = alloc_dev(L, &D.adj_X, (size_t)P.nnz_t * 81)) != LAM_OK) return st;
  if ((st = alloc_dev(L, &p, 1)) != LAM_OK) return st;
  D.adj_flag = reinterpret_cast<int*>(p);  // flag, then emax
  D.adj_ready = true;
  return LAM_OK;
}

template <bool LOWRANK, bool DF, bool SHELL = false>
static lam_status launch_adj_ply(const Plan& P, const AdjArgs& a, cudaStream_t s) {
  const size_t smem = adj_smem(P);
  LAM_CUDA(cudaFuncSetAttribute(adj_ply<LOWRANK, DF, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  dim3 grid((unsigned)adj_nchunks(P), (unsigned)P.plies.size());
  adj_ply<LOWRANK, DF, SHELL><<<grid, adj_block(P), smem, s>>>(a);
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

template <typename Idx, bool SHELL = false>
static lam_status launch_adj_df(const Plan& P, const AdjArgs& a, cudaStream_t s) {
  const size_t smem = adj_df_smem(adj_block(P), sizeof(Idx));
  LAM_CUDA(cudaFuncSetAttribute(adj_ply_df<Idx, SHELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)adj_nchunks(P), (unsigned)P.plies.size());
  adj_ply_df<Idx, SHELL><<<grid, adj_block(P), smem, s>>>(a);
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

// Assembled in-plane Gram blocks (unscaled) into the adjoint workspace G, with
// the maxima of |G_ab| (K-a must have run on the stream).
static lam_status gather_gram(Plan& P, cudaStream_t s) {
  Device& D = *P.dev;
  LAM_CUDA(cudaMemsetAsync(D.adj_gmax, 0, 9 * sizeof(unsigned long long), s));
  AdjGatherArgs g{};
  g.nx = P.u.n;
  g.nel_u = P.u.nel;
  g.nlx = P.u.p + 1;
  g.nls = ka_nls(P);
  g.npl = ka_npl(P);
  g.LSb = D.LSb;
  g.lenX = D.lenX;
  g.lenY = D.lenY;
  g.loX = D.loX;
  g.loY = D.loY;
  g.eloX = D.eloX;
  g.ehiX = D.ehiX;
  g.eloY = D.eloY;
  g.ehiY = D.ehiY;
  g.firstU = D.firstU;
  g.firstV = D.firstV;
  g.EG = D.EG;
  g.G = D.adj_G;
  g.gmax = D.adj_gmax;
  adj_gather<<<(unsigned)P.ns, adj_block(P), 0, s>>>(g);
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

// General extrusion: every (a, b) of D_l meets all four thickness types. The
// 6 x 6 Gram blocks (assembled on the first call and kept) are multiplied by
// the Q types' scales and divided by one power of two per (a, b), so the
// double-float pass (CSR cotangents) and the FP64 pass accumulate in the same
// units and the reduce restores them with the 9 scales.
static lam_status adjoint_shell(Plan& P, const lam_cotangent& cot, double* dC, double* dtheta, double* dDout,
                                cudaStream_t s) {
  Device& D = *P.dev;
  lam_status st;
  if (!D.adj_g_cached) {
    const int64_t n36 = 36 * P.nnz_s;
    if (!D.adj_G36 && (st = alloc_dev(D.allocs, &D.adj_G36, (size_t)n36)) != LAM_OK) return st;
    if (!D.adj_G36df) {
      double* p = nullptr;
      if ((st = alloc_dev(D.allocs, &p, (size_t)n36)) != LAM_OK) return st;
      D.adj_G36df = reinterpret_cast<float2*>(p);
    }
    if (!D.adj_gscale36 && (st = alloc_dev(D.allocs, &D.adj_gscale36, 9)) != LAM_OK) return st;
    if ((st = shell_element_gram(P, s)) != LAM_OK) return st;
    cudaEvent_t ev0 = prof_begin(P, s);
    kg_shell<<<(unsigned)P.ns, 256, 0, s>>>(kp_shell_args(P), D.adj_G36);
    LAM_CUDA(cudaGetLastError());
    const double* q = P.adj_qscale;
    LAM_CUDA(cudaMemsetAsync(D.adj_gmax, 0, 9 * sizeof(unsigned long long), s));
    const unsigned grid = (unsigned)std::min<int64_t>((n36 + 255) / 256, 152 * 8);
    kg_shell_max<<<grid, 256, 0, s>>>(n36, D.adj_G36, q[0], q[1], q[2], q[3], D.adj_gmax);
    LAM_CUDA(cudaGetLastError());
    kg_shell_split<<<grid, 256, 0, s>>>(n36, D.adj_G36, q[0], q[1], q[2], q[3], D.adj_gmax, D.adj_G36df,
                                        D.adj_gscale36);
    LAM_CUDA(cudaGetLastError());
    prof_end(P, LAM_KERNEL_ADJOINT_AUX, 3, s, ev0);
    D.adj_g_cached = true;
  }
  LAM_CUDA(cudaMemsetAsync(D.adj_flag, 0, 2 * sizeof(int), s));
  AdjArgs a{};
  a.ns = P.ns;
  a.n_dof = P.n_dof;
  a.nx = P.u.n;
  a.lsp = max_len_s(P);
  a.nchunks = adj_nchunks(P);
  a.mt = P.adj_max_terms;
  a.LSb = D.LSb;
  a.lenX = D.lenX;
  a.lenY = D.lenY;
  a.loX = D.loX;
  a.loY = D.loY;
  a.term_begin = D.adj_begin;
  a.term_pair = D.adj_pair;
  a.term_q = D.adj_q;
  a.term_qdf = D.adj_qdf;
  a.tp_A = D.tp_A;
  a.tp_lt = D.tp_lt;
  a.tp_k = D.tp_k;
  a.tp_row = D.tp_row;
  a.tp_col = D.tp_col;
  a.gbar = cot.values;
  a.u = cot.u;
  a.v = cot.v;
  a.rank = cot.rank;
  a.G36 = D.adj_G36;      // already multiplied by qs[type] / gscale[ab]
  for (int k = 0; k < 4; ++k) a.qs[k] = 1.0;
  a.G36df = D.adj_G36df;
  a.partial = D.adj_partial;
  a.flag = D.adj_flag;
  a.emax = D.adj_flag + 1;
  const bool lowrank = cot.kind == LAM_COTANGENT_LOWRANK;
  const bool want_df = (cot.flags & LAM_ADJOINT_DOUBLE_FLOAT) != 0;
  // double-float pass (opt-in) for CSR cotangents whose plies meet few
  // thickness pairs; the FP64 pass after it runs only when its result is rejected
  const bool df = !lowrank && want_df && P.adj_max_terms <= kAdjFastTerms;
  cudaEvent_t ev = prof_begin(P, s);
  if (df) {
    a.conditional = 0;
    st = P.nnz < ((int64_t)1 << 31) ? launch_adj_df<int32_t, true>(P, a, s) : launch_adj_df<int64_t, true>(P, a, s);
    if (st != LAM_OK) return st;
    prof_end(P, LAM_KERNEL_ADJOINT, 1, s, ev);
    ev = prof_begin(P, s);
  }
  a.conditional = df ? 1 : 0;
  st = lowrank ? launch_adj_ply<true, false, true>(P, a, s) : launch_adj_ply<false, false, true>(P, a, s);
  if (st != LAM_OK) return st;
  int aux = 1;
  if (df) {
    ++aux;  // the conditional FP64 pass
  } else {
    prof_end(P, LAM_KERNEL_ADJOINT, 1, s, ev);
    ev = prof_begin(P, s);
  }
  AdjReduceArgs r{};
  r.nchunks = a.nchunks;
  for (int k = 0; k < 4; ++k) r.qscale[k] = 1.0;
  r.gscale = D.adj_gscale36;
  r.partial = D.adj_partial;
  r.ply_M = D.ply_M;
  r.ply_dM = D.ply_dM;
  r.mat_C = D.mat_C;
  r.ply_mat = D.ply_mat;
  r.dD = dDout;
  r.dtheta = dtheta;
  r.plyC = D.adj_plyC;
  adj_reduce<<<(unsigned)P.plies.size(), 384, 0, s>>>(r);
  LAM_CUDA(cudaGetLastError());
  if (dC) {
    adj_material<<<1, 256, 0, s>>>((int)P.plies.size(), (int)P.mats.size(), D.ply_mat, D.adj_plyC, dC);
    LAM_CUDA(cudaGetLastError());
    ++aux;
  }
  prof_end(P, LAM_KERNEL_ADJOINT_AUX, aux, s, ev);
  return LAM_OK;
}

static lam_status adjoint(Plan& P, const lam_cotangent& cot, double* dC, double* dtheta, double* dDout,
                          cudaStream_t s) {
  if (P.shell) return adjoint_shell(P, cot, dC, dtheta, dDout, s);
  Device& D = *P.dev;
  lam_status st;
  double* gscale = reinterpret_cast<double*>(D.adj_gmax + 9);
  cudaEvent_t ev;
  if (!D.adj_g_cached) {
    // the in-plane Gram blocks depend on the geometry only, which a plan never
    // changes: computed on the first call and kept
    if ((st = inplane_gram(P, s)) != LAM_OK) return st;
    ev = prof_begin(P, s);
    if ((st = gather_gram(P, s)) != LAM_OK) return st;
    const int64_t n9 = 9 * P.nnz_s;
    adj_split<<<(unsigned)std::min<int64_t>((n9 + 255) / 256, 152 * 8), 256, 0, s>>>(n9, D.adj_G, D.adj_Gdf,
                                                                                      D.adj_gmax, gscale);
    LAM_CUDA(cudaGetLastError());
    prof_end(P, LAM_KERNEL_ADJOINT_AUX, 2, s, ev);
    D.adj_g_cached = true;
  }
  LAM_CUDA(cudaMemsetAsync(D.adj_flag, 0, 2 * sizeof(int), s));
  AdjArgs a{};
  a.ns = P.ns;
  a.n_dof = P.n_dof;
  a.nx = P.u.n;
  a.lsp = max_len_s(P);
  a.nchunks = adj_nchunks(P);
  a.mt = P.adj_max_terms;
  a.LSb = D.LSb;
  a.lenX = D.lenX;
  a.lenY = D.lenY;
  a.loX = D.loX;
  a.loY = D.loY;
  a.term_begin = D.adj_begin;
  a.term_pair = D.adj_pair;
  a.term_q = D.adj_q;
  a.term_qdf = D.adj_qdf;
  a.tp_A = D.tp_A;
  a.tp_lt = D.tp_lt;
  a.tp_k = D.tp_k;
  a.tp_row = D.tp_row;
  a.tp_col = D.tp_col;
  a.gbar = cot.values;
  a.u = cot.u;
  a.v = cot.v;
  a.rank = cot.rank;
  a.G = D.adj_G;
  a.Gdf = D.adj_Gdf;
  a.partial = D.adj_partial;
  a.flag = D.adj_flag;
  a.emax = D.adj_flag + 1;
  const bool lowrank = cot.kind == LAM_COTANGENT_LOWRANK;
  // LAM_ADJOINT_FP64 sends a low-rank cotangent through the generic FP64 pass
  // (a cross-check of the factorised one); LAM_ADJOINT_DOUBLE_FLOAT opts a CSR
  // cotangent into the double-float pass
  const bool force64 = (cot.flags & LAM_ADJOINT_FP64) != 0;
  const bool df = !lowrank && (cot.flags & LAM_ADJOINT_DOUBLE_FLOAT) != 0;
  int nchunks_out = a.nchunks;
  ev = prof_begin(P, s);
  if (lowrank && !force64) {
    // factorised form, FP64 throughout
    AdjLrArgs lr{};
    lr.ns = P.ns;
    lr.nt = P.nt;
    lr.n_dof = P.n_dof;
    lr.nx = P.u.n;
    lr.LSb = D.LSb;
    lr.lenX = D.lenX;
    lr.lenY = D.lenY;
    lr.loX = D.loX;
    lr.loY = D.loY;
    lr.G = D.adj_G;
    lr.W = D.adj_W;
    lr.X = D.adj_X;
    lr.npairs = P.nnz_t;
    lr.tp_row = D.tp_row;
    lr.tp_col = D.tp_col;
    const int64_t nw = P.nt * P.ns * 27;
    for (int q = 0; q < cot.rank; ++q) {
      lr.u = cot.u + (size_t)q * P.n_dof;
      lr.v = cot.v + (size_t)q * P.n_dof;
      lr.accumulate = q > 0;
      adj_lr_w<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(lr);
      LAM_CUDA(cudaGetLastError());
      adj_lr_x<<<(unsigned)P.nnz_t, 256, 0, s>>>(lr);
      LAM_CUDA(cudaGetLastError());
    }
    adj_lr_ply<<<(unsigned)P.plies.size(), 96, 0, s>>>(D.adj_begin, D.adj_pair, D.adj_q, D.adj_X, D.adj_partial);
    LAM_CUDA(cudaGetLastError());
    prof_end(P, LAM_KERNEL_ADJOINT, 2 * cot.rank + 1, s, ev);
    ev = prof_begin(P, s);
    nchunks_out = 1;
  } else if (df) {
    a.conditional = 0;
    if (P.adj_max_terms > kAdjFastTerms)
      st = launch_adj_ply<false, true>(P, a, s);
    else if (P.nnz < ((int64_t)1 << 31))
      st = launch_adj_df<int32_t>(P, a, s);
    else
      st = launch_adj_df<int64_t>(P, a, s);
    if (st != LAM_OK) return st;
    prof_end(P, LAM_KERNEL_ADJOINT, 1, s, ev);
    ev = prof_begin(P, s);
  }
  int aux = 1;  // the reduce
  if (!(lowrank && !force64)) {
    a.conditional = df ? 1 : 0;  // after a double-float pass it runs only when that result is rejected
    st = lowrank ? launch_adj_ply<true, false>(P, a, s) : launch_adj_ply<false, false>(P, a, s);
    if (st != LAM_OK) return st;
    if (!df) {
      prof_end(P, LAM_KERNEL_ADJOINT, 1, s, ev);
      ev = prof_begin(P, s);
    } else {
      ++aux;  // the conditional FP64 pass
    }
  }
  AdjReduceArgs r{};
  r.nchunks = nchunks_out;
  for (int k = 0; k < 4; ++k) r.qscale[k] = P.adj_qscale[k];
  r.gscale = gscale;
  r.partial = D.adj_partial;
  r.ply_M = D.ply_M;
  r.ply_dM = D.ply_dM;
  r.mat_C = D.mat_C;
  r.ply_mat = D.ply_mat;
  r.dD = dDout;
  r.dtheta = dtheta;
  r.plyC = D.adj_plyC;
  adj_reduce<<<(unsigned)P.plies.size(), 384, 0, s>>>(r);
  LAM_CUDA(cudaGetLastError());
  if (dC) {
    adj_material<<<1, 256, 0, s>>>((int)P.plies.size(), (int)P.mats.size(), D.ply_mat, D.adj_plyC, dC);
    LAM_CUDA(cudaGetLastError());
    ++aux;
  }
  prof_end(P, LAM_KERNEL_ADJOINT_AUX, aux, s, ev);
  return LAM_OK;
}

// ---------------------------------------------------------------------------
// In-plane operators of Eq. P (lam_inplane_operators), two constructions.
// Block k of P (11, 12, 21, 22) pairs the derivative / value parts: with
// A_1 = {x, y} and A_2 = {z} (g_z = S), P_k[c][d] = sum_{a in A_alpha, b in
// A_beta} D[V(c,a)][V(d,b)] G_ab for the Gram-block construction.
// ---------------------------------------------------------------------------
__global__ void kp_from_gram(int64_t nps, const double* __restrict__ G, const double* __restrict__ E,
                             double* __restrict__ P) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nps * 36) return;
  const int64_t ps = t / 36;
  const int k = (int)(t % 36), blk = k / 9, cd = k % 9;
  const int a0 = (blk < 2) ? 0 : 2, a1 = (blk < 2) ? 1 : 2;  // A_alpha
  const int b0 = (blk % 2 == 0) ? 0 : 2, b1 = (blk % 2 == 0) ? 1 : 2;
  double acc = 0.0;
  for (int a = a0; a <= a1; ++a)
    for (int b = b0; b <= b1; ++b) acc += E[cd * 9 + a * 3 + b] * G[ps * 9 + a * 3 + b];
  P[t] = acc;
}

// Appendix A, per in-plane element: at every Gauss point the contracted
// tensors C~_ab[p][r] = sum_{i,j} C{e_i, e_j}_{pr} (g^i . e_a)(g^j . e_b), with
// g^i . e_a = (DF^{-1})_{ai} (block-diagonal for the planar map with dz/dxi3 = 1,
// full for a general extrusion, Eq. extrusion),
// and the parametric gradients of the in-plane functions; thread per ordered
// local pair accumulates the four blocks. EP[e][li * nls + lj][36].
struct BfreeArgs {
  InplaneArgs ip;
  const double* Cb;  // [i][j][p][r] of one configuration
  double* EP;
};

__global__ void __launch_bounds__(256) kp_bfree(BfreeArgs a) {
  extern __shared__ double sm[];
  const InplaneArgs& ip = a.ip;
  const int nlx = ip.pu + 1, nly = ip.pv + 1, nls = nlx * nly, nqs = ip.nqu * ip.nqv;
  const int e = blockIdx.x, ex = e % ip.nel_u, ey = e / ip.nel_u;
  const int fx = ip.firstU[ex], fy = ip.firstV[ey];
  double* sS = sm;                              // [q][k] value
  double* sSu = sS + (size_t)nqs * nls;         // d/dxi1
  double* sSv = sSu + (size_t)nqs * nls;        // d/dxi2
  double* sCt = sSv + (size_t)nqs * nls;        // [q][a*3+b][p*3+r]
  double* sJ = sCt + (size_t)nqs * 81;          // [q][16]: rows of DF^-1 (9), w |DF|, W, W1, W2
  // geometry per point
  for (int t = threadIdx.x; t < nqs; t += blockDim.x) {
    const int qu = t % ip.nqu, qv = t / ip.nqu;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2;
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2;
    double W = 1.0, W1 = 0.0, W2 = 0.0;
    if (ip.weights) {
      W = 0.0;
      for (int ly = 0; ly < nly; ++ly)
        for (int lx = 0; lx < nlx; ++lx) {
          const double w = ip.weights[(size_t)(fy + ly) * ip.nx + fx + lx];
          const double wu = w * tu[2 * lx], wdu = w * tu[2 * lx + 1];  // explicit FMAs: same rounding in every kernel
          W = fma(wu, tv[2 * ly], W);
          W1 = fma(wdu, tv[2 * ly], W1);
          W2 = fma(wu, tv[2 * ly + 1], W2);
        }
    }
    // DF = [dS/dxi1 | dS/dxi2 | a] (columns A0, A1, a); planar: S = (x, y, 0), a = e_z
    double A0[3] = {0.0, 0.0, 0.0}, A1[3] = {0.0, 0.0, 0.0};
    for (int ly = 0; ly < nly; ++ly)
      for (int lx = 0; lx < nlx; ++lx) {
        const size_t gi = (size_t)(fy + ly) * ip.nx + fx + lx;
        const double N = tu[2 * lx] * tv[2 * ly], N1 = tu[2 * lx + 1] * tv[2 * ly], N2 = tu[2 * lx] * tv[2 * ly + 1];
        double R1 = N1, R2 = N2;
        if (ip.weights) {
          const double w = ip.weights[gi];
          R1 = w * (N1 * W - N * W1) / (W * W);
          R2 = w * (N2 * W - N * W2) / (W * W);
        }
        if (ip.ctrl3) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            A0[c] += R1 * ip.ctrl3[3 * gi + c];
            A1[c] += R2 * ip.ctrl3[3 * gi + c];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            A0[c] += R1 * ip.ctrl[2 * gi + c];
            A1[c] += R2 * ip.ctrl[2 * gi + c];
          }
        }
      }
    double* d = sJ + (size_t)t * 16;
    double det;
    if (ip.ctrl3) {  // the dual vectors g^k (rows of DF^-1), as in shell_points
      const double A2[3] = {ip.ax, ip.ay, ip.az};
      double g0[3], g1[3], g2[3];
      cross3(A1, A2, g0);
      cross3(A2, A0, g1);
      cross3(A0, A1, g2);
      det = A0[0] * g0[0] + A0[1] * g0[1] + A0[2] * g0[2];
      const double inv = 1.0 / det;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[c] = g0[c] * inv;
        d[3 + c] = g1[c] * inv;
        d[6 + c] = g2[c] * inv;
      }
    } else {
      det = A0[0] * A1[1] - A1[0] * A0[1];
      const double inv = 1.0 / det;
      d[0] = A1[1] * inv;   // (DF^-1)_{00}
      d[1] = -A1[0] * inv;  // (DF^-1)_{01}
      d[2] = 0.0;
      d[3] = -A0[1] * inv;  // (DF^-1)_{10}
      d[4] = A0[0] * inv;   // (DF^-1)_{11}
      d[5] = 0.0;
      d[6] = 0.0;
      d[7] = 0.0;
      d[8] = 1.0;
    }
    d[9] = ip.wU[(size_t)ex * ip.nqu + qu] * ip.wV[(size_t)ey * ip.nqv + qv] * fabs(det);
    d[10] = W;
    d[11] = W1;
    d[12] = W2;
  }
  __syncthreads();
  // parametric values and derivatives of the local functions
  for (int t = threadIdx.x; t < nqs * nls; t += blockDim.x) {
    const int q = t / nls, k = t % nls;
    const int qu = q % ip.nqu, qv = q / ip.nqu, lx = k % nlx, ly = k / nlx;
    const double* tu = ip.tabU + ((size_t)ex * ip.nqu + qu) * nlx * 2;
    const double* tv = ip.tabV + ((size_t)ey * ip.nqv + qv) * nly * 2;
    double R = tu[2 * lx] * tv[2 * ly], R1 = tu[2 * lx + 1] * tv[2 * ly], R2 = tu[2 * lx] * tv[2 * ly + 1];
    if (ip.weights) {
      const double* d = sJ + (size_t)q * 16;
      const double w = ip.weights[(size_t)(fy + ly) * ip.nx + fx + lx], W = d[10];
      const double N = R, N1 = R1, N2 = R2;
      R = w * N / W;
      R1 = w * (N1 * W - N * d[11]) / (W * W);
      R2 = w * (N2 * W - N * d[12]) / (W * W);
    }
    sS[t] = R;
    sSu[t] = R1;
    sSv[t] = R2;
  }
  // contracted tensors
  for (int t = threadIdx.x; t < nqs * 81; t += blockDim.x) {
    const int q = t / 81, ab = (t % 81) / 9, pr = t % 9;
    const int al = ab / 3, be = ab % 3;
    const double* d = sJ + (size_t)q * 16;
    double gi[3], gj[3];  // (DF^-1)_{alpha i}, (DF^-1)_{beta j}
    for (int i = 0; i < 3; ++i) {
      gi[i] = d[al * 3 + i];
      gj[i] = d[be * 3 + i];
    }
    double acc = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) acc += a.Cb[(i * 3 + j) * 9 + pr] * gi[i] * gj[j];
    sCt[t] = acc;
  }
  __syncthreads();
  for (int pair = threadIdx.x; pair < nls * nls; pair += blockDim.x) {
    const int li = pair / nls, lj = pair % nls;
    double acc[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) acc[k] = 0.0;
    for (int q = 0; q < nqs; ++q) {
      const double w = sJ[(size_t)q * 16 + 9];
      const double Si = sS[q * nls + li], Sj = sS[q * nls + lj];
      const double Ui = sSu[q * nls + li], Uj = sSu[q * nls + lj];
      const double Vi = sSv[q * nls + li], Vj = sSv[q * nls + lj];
      const double* C = sCt + (size_t)q * 81;
      const double f00 = w * Ui * Uj, f01 = w * Ui * Vj, f10 = w * Vi * Uj, f11 = w * Vi * Vj;
      const double f02 = w * Ui * Sj, f12 = w * Vi * Sj, f20 = w * Si * Uj, f21 = w * Si * Vj, f22 = w * Si * Sj;
#pragma unroll
      for (int pr = 0; pr < 9; ++pr) {
        acc[pr] += C[0 * 9 + pr] * f00 + C[1 * 9 + pr] * f01 + C[3 * 9 + pr] * f10 + C[4 * 9 + pr] * f11;
        acc[9 + pr] += C[2 * 9 + pr] * f02 + C[5 * 9 + pr] * f12;
        acc[18 + pr] += C[6 * 9 + pr] * f20 + C[7 * 9 + pr] * f21;
        acc[27 + pr] += C[8 * 9 + pr] * f22;
      }
    }
    double* out = a.EP + ((size_t)e * nls * nls + pair) * 36;
#pragma unroll
    for (int k = 0; k < 36; ++k) out[k] = acc[k];
  }
}

// Sum of the element operators over the elements an in-plane pair shares.
struct PGatherArgs {
  int nx, nel_u, nlx, nls;
  const int64_t* LSb;
  const int *lenX, *lenY, *loX, *loY, *eloX, *ehiX, *eloY, *ehiY, *firstU, *firstV;
  const double* EP;
  double* P;
};

__global__ void kp_gather(PGatherArgs a) {
  const int64_t is = blockIdx.x;
  const int ix = (int)(is % a.nx), iy = (int)(is / a.nx);
  const int lx = a.lenX[ix], ls = lx * a.lenY[iy];
  const int64_t ls0 = a.LSb[is];
  for (int item = threadIdx.x; item < 36 * ls; item += blockDim.x) {
    const int ks = item / 36, k = item % 36;
    const int jx = a.loX[ix] + ks % lx, jy = a.loY[iy] + ks / lx;
    const int ex0 = max(a.eloX[ix], a.eloX[jx]), ex1 = min(a.ehiX[ix], a.ehiX[jx]);
    const int ey0 = max(a.eloY[iy], a.eloY[jy]), ey1 = min(a.ehiY[iy], a.ehiY[jy]);
    double acc = 0.0;
    for (int ey = ey0; ey <= ey1; ++ey) {
      const int fy = a.firstV[ey];
      for (int ex = ex0; ex <= ex1; ++ex) {
        const int fx = a.firstU[ex];
        const int li = (iy - fy) * a.nlx + (ix - fx), lj = (jy - fy) * a.nlx + (jx - fx);
        acc += a.EP[(((size_t)ey * a.nel_u + ex) * a.nls * a.nls + (size_t)li * a.nls + lj) * 36 + k];
      }
    }
    a.P[(ls0 + ks) * 36 + k] = acc;
  }
}

static lam_status pattern_args(const Plan& P, PatArgs& a) {
  const Device& D = *P.dev;
  a.ns = P.ns;
  a.nt = P.nt;
  a.n_dof = P.n_dof;
  a.nnz = P.nnz;
  a.nnz_s = P.nnz_s;
  a.nx = P.u.n;
  a.LSb = D.LSb;
  a.LTb = D.LTb;
  a.loX = D.loX;
  a.lenX = D.lenX;
  a.loY = D.loY;
  a.lenY = D.lenY;
  a.loT = D.loT;
  a.lenT = D.lenT;
  return LAM_OK;
}

}  // namespace lam

// ---------------------------------------------------------------------------
// Device C ABI
// ---------------------------------------------------------------------------
extern "C" {

lam_status lam_plan_destroy(lam_plan* plan) {
  if (!plan) return LAM_OK;
  lam::free_device(plan->p);
  delete plan;
  return LAM_OK;
}

lam_status lam_pattern(lam_plan* plan, int64_t* nnz_out, int64_t* d_row_ptr, int32_t* d_col_ind, void* stream) {
  if (!plan) {
    lam::set_error("lam_pattern: plan is NULL");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  if (nnz_out) *nnz_out = P.nnz;
  if (!d_row_ptr && !d_col_ind) return LAM_OK;
  if (!d_row_ptr || !d_col_ind) {
    lam::set_error("lam_pattern: give both d_row_ptr and d_col_ind, or neither");
    return LAM_ERR_INVALID_ARG;
  }
  lam_status st = lam::ensure_device(P);
  if (st != LAM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lam::PatArgs a;
  lam::pattern_args(P, a);
  const int64_t rows = P.n_dof + 1;
  cudaEvent_t ev = lam::prof_begin(P, s);
  lam::kp_row_ptr<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(a, d_row_ptr);
  LAM_CUDA(cudaGetLastError());
  dim3 grid((unsigned)P.ns, (unsigned)P.nt);
  lam::kp_col_ind<<<grid, 256, 0, s>>>(a, d_col_ind);
  LAM_CUDA(cudaGetLastError());
  lam::prof_end(P, LAM_KERNEL_PATTERN, 2, s, ev);
  return LAM_OK;
}

lam_status lam_assemble_split(lam_plan* plan, double* d_values, void* stream) {
  if (!plan || !d_values) {
    lam::set_error("lam_assemble_split: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  if ((st = lam::ensure_device(P)) != LAM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = lam::split_integrals(P, s)) != LAM_OK) return st;
  lam::KcArgs k = lam::kc_args(P, d_values);
  return lam::launch_combine<false>(P, k, s);
}

lam_status lam_assemble_split_host(lam_plan* plan, double* h_values, void* stream) {
  if (!plan || !h_values) {
    lam::set_error("lam_assemble_split_host: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  if ((st = lam::ensure_device(P)) != LAM_OK) return st;
  lam::Device& D = *P.dev;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // slabs of thickness rows: at least about 256 MB of values each and at most
  // about twelve slabs (every slab's combine forms the slices of all of its
  // rows' classes, so fewer slabs cost less arithmetic; the first slab's
  // kernels and the last slab's copy are not overlapped)
  const int64_t per_row = 9 * P.nnz_s * 4;  // upper bound of one thickness row's share (len_t <= 4 avg)
  int64_t rows_per_slab = std::max<int64_t>(1, (int64_t)(32 << 20) / std::max<int64_t>(1, per_row));
  rows_per_slab = std::max<int64_t>(rows_per_slab, (P.nt + 11) / 12);
  rows_per_slab = std::min<int64_t>(rows_per_slab, P.nt);
  size_t need = 0;
  for (int64_t r0 = 0; r0 < P.nt; r0 += rows_per_slab) {
    const int64_t r1 = std::min<int64_t>(P.nt, r0 + rows_per_slab);
    need = std::max<size_t>(need, (size_t)(9 * (P.LTb[r1] - P.LTb[r0]) * P.nnz_s));
  }
  if (D.stage_elems < need) {
    for (int k = 0; k < 2; ++k) {
      if (D.stage[k]) cudaFree(D.stage[k]);
      D.stage[k] = nullptr;
      cudaError_t e = lam::device_alloc(reinterpret_cast<void**>(&D.stage[k]), need * sizeof(double));
      if (e != cudaSuccess) {
        lam::set_error("cudaMalloc(staging) failed: %s", cudaGetErrorString(e));
        D.stage_elems = 0;
        return LAM_ERR_OOM;
      }
    }
    D.stage_elems = need;
  }
  if (!D.copy_stream) {
    LAM_CUDA(cudaStreamCreateWithFlags(&D.copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      LAM_CUDA(cudaEventCreateWithFlags(&D.ev_done[k], cudaEventDisableTiming));
      LAM_CUDA(cudaEventCreateWithFlags(&D.ev_copied[k], cudaEventDisableTiming));
      LAM_CUDA(cudaEventRecord(D.ev_copied[k], D.copy_stream));
    }
  }
  if ((st = lam::split_integrals(P, s)) != LAM_OK) return st;
  int slot = 0;
  for (int64_t r0 = 0; r0 < P.nt; r0 += rows_per_slab, slot ^= 1) {
    const int64_t r1 = std::min<int64_t>(P.nt, r0 + rows_per_slab);
    const int64_t off = 9 * P.LTb[r0] * P.nnz_s, cnt = 9 * (P.LTb[r1] - P.LTb[r0]) * P.nnz_s;
    LAM_CUDA(cudaStreamWaitEvent(s, D.ev_copied[slot], 0));
    lam::KcArgs k = lam::kc_args(P, D.stage[slot]);
    k.it_lo = (int)r0;
    k.it_hi = (int)r1;
    k.out_offset = off;
    st = lam::launch_combine<true>(P, k, s);
    if (st != LAM_OK) return st;
    LAM_CUDA(cudaEventRecord(D.ev_done[slot], s));
    LAM_CUDA(cudaStreamWaitEvent(D.copy_stream, D.ev_done[slot], 0));
    LAM_CUDA(cudaMemcpyAsync(h_values + off, D.stage[slot], (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost,
                             D.copy_stream));
    P.prof_d2h += cnt * (int64_t)sizeof(double);
    LAM_CUDA(cudaEventRecord(D.ev_copied[slot], D.copy_stream));
  }
  LAM_CUDA(cudaStreamSynchronize(D.copy_stream));
  LAM_CUDA(cudaStreamSynchronize(s));
  return LAM_OK;
}

lam_status lam_assemble_standard(lam_plan* plan, double* d_values, void* stream) {
  if (!plan || !d_values) {
    lam::set_error("lam_assemble_standard: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  if ((st = lam::ensure_device(P)) != LAM_OK) return st;
  lam::Device& D = *P.dev;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LAM_CUDA(cudaMemsetAsync(d_values, 0, (size_t)P.nnz * sizeof(double), s));
  lam::KdArgs k{};
  k.ip = lam::inplane_args(P);
  k.nel_v = P.v.nel;
  k.nqt = P.nqt;
  k.q1 = P.t.p + 1;
  k.ns = P.ns;
  k.nnz_s = P.nnz_s;
  k.loX = D.loX;
  k.lenX = D.lenX;
  k.loY = D.loY;
  k.lenY = D.lenY;
  k.loT = D.loT;
  k.lenT = D.lenT;
  k.firstT = D.firstT;
  k.LSb = D.LSb;
  k.LTb = D.LTb;
  k.piece_begin = D.piece_begin;
  k.piece_cfg = D.piece_cfg;
  k.tabT = D.tabT;
  k.wT = D.wT;
  k.cfgE = D.cfgE;
  k.values = d_values;
  const size_t smem = lam::kd_smem(P);
  LAM_CUDA(cudaFuncSetAttribute(lam::kd_standard<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LAM_CUDA(cudaFuncSetAttribute(lam::kd_standard<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ncol = (int)P.col3_begin.size() - 1;
  cudaEvent_t ev = lam::prof_begin(P, s);
  int launched = 0;
  for (int c = 0; c < ncol; ++c) {
    const int n = P.col3_begin[c + 1] - P.col3_begin[c];
    if (n == 0) continue;
    k.elems = D.col3_elem + P.col3_begin[c];
    if (P.shell)
      lam::kd_standard<true><<<n, 256, smem, s>>>(k);
    else
      lam::kd_standard<false><<<n, 256, smem, s>>>(k);
    LAM_CUDA(cudaGetLastError());
    ++launched;
  }
  lam::prof_end(P, LAM_KERNEL_STANDARD, launched, s, ev);
  return LAM_OK;
}

lam_status lam_adjoint(lam_plan* plan, const lam_cotangent* cot, double* d_dC, double* d_dtheta, double* d_dD,
                       void* stream) {
  if (!plan || !cot) {
    lam::set_error("lam_adjoint: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  if (cot->kind == LAM_COTANGENT_CSR) {
    if (!cot->values) {
      lam::set_error("lam_adjoint: CSR cotangent without values");
      return LAM_ERR_INVALID_ARG;
    }
  } else if (cot->kind == LAM_COTANGENT_LOWRANK) {
    if (cot->rank < 1 || !cot->u || !cot->v) {
      lam::set_error("lam_adjoint: low-rank cotangent needs rank >= 1 and both u and v");
      return LAM_ERR_INVALID_ARG;
    }
  } else {
    lam::set_error("lam_adjoint: unknown cotangent kind %d", (int)cot->kind);
    return LAM_ERR_INVALID_ARG;
  }
  if ((cot->flags & ~(LAM_ADJOINT_FP64 | LAM_ADJOINT_DOUBLE_FLOAT)) != 0 ||
      (cot->flags & (LAM_ADJOINT_FP64 | LAM_ADJOINT_DOUBLE_FLOAT)) == (LAM_ADJOINT_FP64 | LAM_ADJOINT_DOUBLE_FLOAT)) {
    lam::set_error("lam_adjoint: unknown or conflicting flags 0x%x", (unsigned)cot->flags);
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  if (P.adj_max_terms > lam::kAdjMaxTerms) {
    lam::set_error("lam_adjoint: a ply meets %d thickness pairs (at most %d)", P.adj_max_terms, lam::kAdjMaxTerms);
    return LAM_ERR_UNSUPPORTED;
  }
  if (!d_dC && !d_dtheta && !d_dD) return LAM_OK;
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  if ((st = lam::ensure_device(P)) != LAM_OK) return st;
  if ((st = lam::ensure_adjoint(P)) != LAM_OK) return st;
  return lam::adjoint(P, *cot, d_dC, d_dtheta, d_dD, static_cast<cudaStream_t>(stream));
}

lam_status lam_inplane_operators(lam_plan* plan, int32_t ply, int32_t method, double* d_P, void* stream) {
  if (!plan || !d_P) {
    lam::set_error("lam_inplane_operators: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  if (ply < 0 || ply >= (int32_t)P.plies.size()) {
    lam::set_error("lam_inplane_operators: ply %d of %d", ply, (int)P.plies.size());
    return LAM_ERR_INVALID_ARG;
  }
  if (method != LAM_P_FROM_GRAM && method != LAM_P_VOIGT_FREE) {
    lam::set_error("lam_inplane_operators: unknown method %d", method);
    return LAM_ERR_INVALID_ARG;
  }
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  if ((st = lam::ensure_device(P)) != LAM_OK) return st;
  lam::Device& D = *P.dev;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int m = P.ply_cfg[ply];
  if (method == LAM_P_FROM_GRAM && P.shell) {  // the 6 x 6 Gram blocks and P of every configuration
    if ((st = lam::shell_operators(P, s, true)) != LAM_OK) return st;
    LAM_CUDA(cudaMemcpyAsync(d_P, D.shellP + (size_t)m * P.nnz_s * 36, (size_t)P.nnz_s * 36 * sizeof(double),
                             cudaMemcpyDeviceToDevice, s));
    return LAM_OK;
  }
  if (method == LAM_P_FROM_GRAM) {
    if ((st = lam::ensure_adjoint(P)) != LAM_OK) return st;
    if ((st = lam::inplane_gram(P, s)) != LAM_OK) return st;
    D.adj_g_cached = false;  // the adjoint's scaled copy is overwritten here
    if ((st = lam::gather_gram(P, s)) != LAM_OK) return st;
    const int64_t n = P.nnz_s * 36;
    lam::kp_from_gram<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P.nnz_s, D.adj_G, D.cfgE + (size_t)m * 81, d_P);
    LAM_CUDA(cudaGetLastError());
    return LAM_OK;
  }
  const int nls = lam::ka_nls(P), nqs = P.nqu * P.nqv, nel = P.u.nel * P.v.nel;
  if (!D.bfree_EP && (st = lam::alloc_dev(D.allocs, &D.bfree_EP, (size_t)nel * nls * nls * 36)) != LAM_OK) return st;
  lam::BfreeArgs a{};
  a.ip = lam::inplane_args(P);
  a.Cb = D.cfgCb + (size_t)m * 81;
  a.EP = D.bfree_EP;
  const size_t smem = ((size_t)3 * nqs * nls + 81 * (size_t)nqs + 16 * (size_t)nqs) * sizeof(double);
  LAM_CUDA(cudaFuncSetAttribute(lam::kp_bfree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int block = std::min(256, std::max(32, ((nls * nls + 31) / 32) * 32));
  lam::kp_bfree<<<(unsigned)nel, block, smem, s>>>(a);
  LAM_CUDA(cudaGetLastError());
  lam::PGatherArgs g{};
  g.nx = P.u.n;
  g.nel_u = P.u.nel;
  g.nlx = P.u.p + 1;
  g.nls = nls;
  g.LSb = D.LSb;
  g.lenX = D.lenX;
  g.lenY = D.lenY;
  g.loX = D.loX;
  g.loY = D.loY;
  g.eloX = D.eloX;
  g.ehiX = D.ehiX;
  g.eloY = D.eloY;
  g.ehiY = D.ehiY;
  g.firstU = D.firstU;
  g.firstV = D.firstV;
  g.EP = D.bfree_EP;
  g.P = d_P;
  lam::kp_gather<<<(unsigned)P.ns, 256, 0, s>>>(g);
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

lam_status lam_profile_enable(lam_plan* plan, int32_t enable) {
  if (!plan) {
    lam::set_error("lam_profile_enable: plan is NULL");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  if (!P.prof_pending.empty()) lam::prof_collect(P);
  P.prof_enabled = enable != 0;
  for (int k = 0; k < LAM_KERNEL_KINDS; ++k) {
    P.prof_launches[k] = 0;
    P.prof_ms[k] = 0.0;
  }
  P.prof_h2d = 0;
  P.prof_d2h = 0;
  return LAM_OK;
}

lam_status lam_profile_get(lam_plan* plan, lam_profile* out) {
  if (!plan || !out) {
    lam::set_error("lam_profile_get: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  lam::Plan& P = plan->p;
  lam::prof_collect(P);
  out->enabled = P.prof_enabled ? 1 : 0;
  for (int k = 0; k < LAM_KERNEL_KINDS; ++k) {
    out->launches[k] = P.prof_launches[k];
    out->ms[k] = P.prof_ms[k];
  }
  out->h2d_bytes = P.prof_h2d;
  out->d2h_bytes = P.prof_d2h;
  return LAM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Split assembly without allocation (lam_assemble_split_noalloc): the same
// kernels, with every table and workspace placed in one static device array.
// ---------------------------------------------------------------------------
#include <mutex>

namespace lam {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LAM_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
static void* g_noalloc_addr[kNoallocMaxDevices] = {};
static std::mutex g_noalloc_mutex;

// Device address of the static array on the current device. Host code cannot
// use the array's name as a device pointer, so the address is looked up once
// per device (with that device current) and remembered.
static lam_status noalloc_scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) {
    set_error("lam_assemble_split_noalloc: device ordinal %d outside [0, %d)", dev, kNoallocMaxDevices);
    return LAM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("lam_assemble_split_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return LAM_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return LAM_OK;
}

// Fills trep[k] = cls_rep[u] for the terms k of every class u.
__global__ void noalloc_term_rep(const int* __restrict__ term_begin, const int* __restrict__ cls_rep, int ncls,
                                 int* __restrict__ trep) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ncls) return;
  for (int k = term_begin[u]; k < term_begin[u + 1]; ++k) trep[k] = cls_rep[u];
}

// Carves the scratch array into 256-byte aligned slices.
struct ScratchCarver {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

}  // namespace lam

extern "C" lam_status lam_assemble_split_noalloc(const lam_plan* plan, double* d_values, void* stream) {
  if (!plan || !d_values) {
    lam::set_error("lam_assemble_split_noalloc: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  const lam::Plan& P = plan->p;
  if (P.shell) {
    lam::set_error("lam_assemble_split_noalloc: general extrusion maps are not supported");
    return LAM_ERR_UNSUPPORTED;
  }
  lam_status st;
  if ((st = lam::check_limits(P)) != LAM_OK) return st;
  const int ncfg = (int)P.cfg_mat.size();
  // layout (sizes only: base 0)
  lam::ScratchCarver lay{nullptr};
  lay.take<double>(P.tabU.size());
  lay.take<double>(P.tabV.size());
  lay.take<double>(P.wU.size());
  lay.take<double>(P.wV.size());
  lay.take<int>(P.u.first.size());
  lay.take<int>(P.v.first.size());
  lay.take<int>(P.u.lo.size());
  lay.take<int>(P.u.len.size());
  lay.take<int>(P.v.lo.size());
  lay.take<int>(P.v.len.size());
  lay.take<double>(P.ctrl.size());
  lay.take<double>(P.weights.size());
  lay.take<int64_t>(P.LSb.size());
  lay.take<int>(P.col2_elem.size());
  lay.take<int>(P.t.first.size());
  lay.take<double>(P.tabT.size());
  lay.take<double>(P.wT.size());
  lay.take<int>(P.piece_begin.size());
  lay.take<int>(P.pieces.size());
  lay.take<int>(P.tp_row.size());
  lay.take<int>(P.tp_col.size());
  lay.take<int>(P.tp_e0.size());
  lay.take<int>(P.tp_e1.size());
  lay.take<int>(P.cls_term_begin.size());
  lay.take<int>(P.cls_terms.size());
  lay.take<int>(P.cls_occ_begin.size());
  lay.take<int>(P.cls_rep.size());
  lay.take<int>(P.cls_terms.size());
  lay.take<int64_t>(P.occ_A.size());
  lay.take<int>(P.occ_lt.size());
  lay.take<int>(P.occ_k.size());
  lay.take<int>(P.occ_it.size());
  lay.take<double>(P.cfgE.size());
  lay.take<double>((size_t)P.nnz_t * ncfg * 4);
  lay.take<double>((size_t)P.nnz_s * 9);
  if (lay.used > LAM_NOALLOC_SCRATCH_BYTES) {
    lam::set_error("lam_assemble_split_noalloc: this plan needs %zu bytes of scratch, the static array holds %u",
                   lay.used, (unsigned)LAM_NOALLOC_SCRATCH_BYTES);
    return LAM_ERR_UNSUPPORTED;
  }
  int dev = 0;
  LAM_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  if ((st = lam::noalloc_scratch_address(dev, &base)) != LAM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lam::ScratchCarver sc{base};
  // tables: host -> static array (stream-ordered copies)
#define PUT(T, name, vec)                                                                              \
  T* name = sc.take<T>((vec).size());                                                                  \
  if (!(vec).empty())                                                                                  \
    LAM_CUDA(cudaMemcpyAsync(name, (vec).data(), (vec).size() * sizeof(T), cudaMemcpyHostToDevice, s));
  PUT(double, tabU, P.tabU);
  PUT(double, tabV, P.tabV);
  PUT(double, wU, P.wU);
  PUT(double, wV, P.wV);
  PUT(int, firstU, P.u.first);
  PUT(int, firstV, P.v.first);
  PUT(int, loX, P.u.lo);
  PUT(int, lenX, P.u.len);
  PUT(int, loY, P.v.lo);
  PUT(int, lenY, P.v.len);
  PUT(double, ctrl, P.ctrl);
  PUT(double, weights, P.weights);
  PUT(int64_t, LSb, P.LSb);
  PUT(int, col2_elem, P.col2_elem);
  PUT(int, firstT, P.t.first);
  PUT(double, tabT, P.tabT);
  PUT(double, wT, P.wT);
  PUT(int, piece_begin, P.piece_begin);
  int* piece_cfg = sc.take<int>(P.pieces.size());
  if (!P.pieces.empty())  // the cfg field of every Piece, gathered by a strided copy
    LAM_CUDA(cudaMemcpy2DAsync(piece_cfg, sizeof(int), &P.pieces[0].cfg, sizeof(lam::Piece), sizeof(int),
                               P.pieces.size(), cudaMemcpyHostToDevice, s));
  PUT(int, tp_row, P.tp_row);
  PUT(int, tp_col, P.tp_col);
  PUT(int, tp_e0, P.tp_e0);
  PUT(int, tp_e1, P.tp_e1);
  PUT(int, cls_term_begin, P.cls_term_begin);
  PUT(int, cls_terms, P.cls_terms);
  PUT(int, cls_occ_begin, P.cls_occ_begin);
  PUT(int, cls_rep, P.cls_rep);
  int* term_rep = sc.take<int>(P.cls_terms.size());
  PUT(int64_t, occ_A, P.occ_A);
  PUT(int, occ_lt, P.occ_lt);
  PUT(int, occ_k, P.occ_k);
  PUT(int, occ_it, P.occ_it);
  PUT(double, cfgE, P.cfgE);
#undef PUT
  double* q = sc.take<double>((size_t)P.nnz_t * ncfg * 4);
  double* G = sc.take<double>((size_t)P.nnz_s * 9);
  lam::noalloc_term_rep<<<(P.ncls + 127) / 128, 128, 0, s>>>(cls_term_begin, cls_rep, P.ncls, term_rep);
  LAM_CUDA(cudaGetLastError());
  // K-b
  lam::KbArgs kb{};
  kb.npairs = P.nnz_t;
  kb.ncfg = ncfg;
  kb.nqt = P.nqt;
  kb.q1 = P.t.p + 1;
  kb.tp_row = tp_row;
  kb.tp_col = tp_col;
  kb.tp_e0 = tp_e0;
  kb.tp_e1 = tp_e1;
  kb.firstT = firstT;
  kb.piece_begin = piece_begin;
  kb.piece_cfg = piece_cfg;
  kb.tabT = tabT;
  kb.wT = wT;
  kb.q = q;
  lam::kb_thickness<<<(unsigned)((P.nnz_t + 127) / 128), 128, 0, s>>>(kb);
  LAM_CUDA(cudaGetLastError());
  // K-a: G accumulates, so it starts at zero
  LAM_CUDA(cudaMemsetAsync(G, 0, (size_t)P.nnz_s * 9 * sizeof(double), s));
  lam::KaArgs ka{};
  ka.ip.nx = P.u.n;
  ka.ip.nel_u = P.u.nel;
  ka.ip.pu = P.u.p;
  ka.ip.pv = P.v.p;
  ka.ip.nqu = P.nqu;
  ka.ip.nqv = P.nqv;
  ka.ip.tabU = tabU;
  ka.ip.tabV = tabV;
  ka.ip.wU = wU;
  ka.ip.wV = wV;
  ka.ip.ctrl = ctrl;
  ka.ip.weights = P.weights.empty() ? nullptr : weights;
  ka.ip.firstU = firstU;
  ka.ip.firstV = firstV;
  ka.loX = loX;
  ka.lenX = lenX;
  ka.loY = loY;
  ka.lenY = lenY;
  ka.LSb = LSb;
  ka.G = G;
  const size_t ka_sm = lam::ka_smem(P);
  LAM_CUDA(cudaFuncSetAttribute(lam::ka_inplane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ka_sm));
  const int ncol = (int)P.col2_begin.size() - 1;
  for (int c = 0; c < ncol; ++c) {
    const int n = P.col2_begin[c + 1] - P.col2_begin[c];
    if (n == 0) continue;
    ka.elems = col2_elem + P.col2_begin[c];
    lam::ka_inplane<<<n, lam::ka_block(P), ka_sm, s>>>(ka);
    LAM_CUDA(cudaGetLastError());
  }
  // K-c
  lam::KcArgs k{};
  k.ns = P.ns;
  k.nnz_s = P.nnz_s;
  k.nx = P.u.n;
  k.ncfg = ncfg;
  k.ncls = P.ncls;
  k.nterms = (int)P.cls_terms.size();
  k.nocc = (int)P.nnz_t;
  k.gs_cap = lam::kc_gs_cap(P);
  k.LSb = LSb;
  k.lenX = lenX;
  k.lenY = lenY;
  k.G = G;
  k.EG = nullptr;
  k.cfgE = cfgE;
  k.q = q;
  k.cls_term_begin = cls_term_begin;
  k.cls_terms = cls_terms;
  k.cls_occ_begin = cls_occ_begin;
  k.term_rep = term_rep;
  k.occ_A = occ_A;
  k.occ_lt = occ_lt;
  k.occ_k = occ_k;
  k.occ_it = occ_it;
  k.it_lo = 0;
  k.it_hi = (int)P.nt;
  k.out_offset = 0;
  k.values = d_values;
  const size_t kc_sm = lam::kc_smem(P);
  if (P.monoclinic) {
    LAM_CUDA(cudaFuncSetAttribute(lam::kc_combine<true, false, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kc_sm));
    lam::kc_combine<true, false, false><<<(unsigned)P.ns, lam::kc_block(P), kc_sm, s>>>(k);
  } else {
    LAM_CUDA(cudaFuncSetAttribute(lam::kc_combine<false, false, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kc_sm));
    lam::kc_combine<false, false, false><<<(unsigned)P.ns, lam::kc_block(P), kc_sm, s>>>(k);
  }
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

// ===========================================================================
// Batches (lam_batch_*): one launch per stage for many laminates.
// ===========================================================================
namespace lam {

__device__ __forceinline__ int find_slot(const int64_t* prefix, int n, int64_t g) {
  int lo = 0, hi = n;  // prefix[lo] <= g < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Eq. Q for every thickness pair of every instance.
__global__ void kb_batch(const KbArgs* __restrict__ args, const int64_t* __restrict__ prefix, int n) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= prefix[n]) return;
  const int i = find_slot(prefix, n, g);
  kb_pair(args[i], g - prefix[i]);
}

// In-plane Gram blocks of every element of every distinct mesh (DF: the
// double-float K-a, otherwise FP64).
template <bool DF>
__global__ void __launch_bounds__(256) ka_batch(const KaLocalArgs* __restrict__ args, const int64_t* __restrict__ prefix,
                                                int n) {
  extern __shared__ double sm[];
  const int i = find_slot(prefix, n, blockIdx.x);
  if (DF)
    ka_elem(args[i], (int)(blockIdx.x - prefix[i]), sm);
  else
    ka_elem64(args[i], (int)(blockIdx.x - prefix[i]), sm);
}

struct BatchKcArgs {
  const KcArgs* kc;           // per instance
  const int64_t* row_prefix;  // work items (blocks of rows_per_item rows) of the instances in work order, n + 1
  int rows_per_item;          // consecutive in-plane rows of one instance per work item
  const int* order;           // work order -> instance
  const int* mono;            // per instance: monoclinic
  int n;
  unsigned long long* counter;
  int* flags;                 // per instance: FP64 re-pass flag, largest exponent
  double* pcache;             // per CTA: 2 * pcache_cfg * blockDim.x doubles (kcs_row's P of a row)
  int pcache_cfg;             // most configurations of an instance
};

// Persistent combine: CTAs take (instance, in-plane row) items from an atomic
// counter until none are left. DF = true: double-float slices; DF = false and
// COND = true: the FP64 re-pass of the flagged instances only; DF = false and
// COND = false: FP64 for every instance. MONO = true when every instance is
// monoclinic; otherwise each row takes its instance's form.
template <bool MONO, bool DF, bool COND = true>
__global__ void __maxnreg__(64) kc_batch(BatchKcArgs b) {
  extern __shared__ double sm[];
  __shared__ unsigned long long s_item;
  // MONO: the current instance's arguments, in shared memory: the rows' CSR stores
  // cannot alias them there, so they need no reloading and no registers across the
  // stores (mixed batches read them from global memory, as their larger kernel
  // spills more with the copy)
  __shared__ KcArgs s_kc;
  int cur = -1;
  const int64_t total = b.row_prefix[b.n];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1ull);
    __syncthreads();
    const int64_t g = (int64_t)s_item;
    __syncthreads();
    if (g >= total) break;
    const int k = find_slot(b.row_prefix, b.n, g);
    const int inst = b.order[k];
    if (MONO && inst != cur) {  // every thread has left the previous item (the barriers above)
      const int* src = reinterpret_cast<const int*>(b.kc + inst);
      int* dst = reinterpret_cast<int*>(&s_kc);
      for (int w = threadIdx.x; w < (int)(sizeof(KcArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      cur = inst;
    }
    const int64_t r0 = (g - b.row_prefix[k]) * b.rows_per_item;
    const int64_t r1 = min(r0 + b.rows_per_item, MONO ? s_kc.ns : b.kc[inst].ns);
    if (!DF && COND && b.flags[2 * inst] == 0) continue;
    int emax = 0;
    bool bad = false;
    // each instance in the form its single-plan assembly takes (bitwise equal results)
    double* pc = b.pcache + (size_t)blockIdx.x * 2 * b.pcache_cfg * blockDim.x;
    for (int64_t r = r0; r < r1; ++r) {
      if (MONO)
        kcs_row<true, false, DF>(s_kc, r, sm, emax, bad, pc);
      else if (b.mono[inst])
        kcs_row<true, false, DF>(b.kc[inst], r, sm, emax, bad, pc);
      else
        kcs_row<false, false, DF>(b.kc[inst], r, sm, emax, bad, pc);
    }
    if (DF) {
      emax = __reduce_max_sync(0xffffffffu, emax);
      const bool any_bad = __any_sync(0xffffffffu, bad);
      if ((threadIdx.x & 31) == 0) {
        atomicMax(&b.flags[2 * inst + 1], emax);
        if (any_bad) atomicOr(&b.flags[2 * inst], 1);
      }
    }
  }
}

__global__ void kc_batch_check(int* flags, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flags[2 * i + 1] < kKcMinExp) flags[2 * i] = 1;
}

}  // namespace lam

struct lam_batch {
  std::vector<lam_plan*> plans;
  std::vector<int> versions;
  int device = -1;
  int n_meshes = 0;
  int64_t nnz_total = 0;
  std::vector<int> persistent;    // instances of the persistent combine (index into plans)
  std::vector<int> fallback;      // instances assembled by lam_assemble_split
  std::vector<int> inst_slot;     // plan -> index in persistent, or -1
  std::vector<void*> allocs;
  // launch tables
  lam::KbArgs* d_kb = nullptr;
  int64_t* d_pair_prefix = nullptr;
  int64_t total_pairs = 0;
  lam::KaLocalArgs* d_ka = nullptr;
  int64_t* d_elem_prefix = nullptr;
  int64_t total_elems = 0;
  lam::KcArgs* d_kc = nullptr;
  lam::KcArgs* h_kc = nullptr;    // pinned host copy (value pointers change per call)
  int64_t* d_row_prefix[3] = {nullptr, nullptr, nullptr};  // work items of 1, 2 and 4 rows
  int* d_order = nullptr;
  int* d_mono = nullptr;
  int* d_flags = nullptr;
  unsigned long long* d_counter = nullptr;
  double* d_pcache = nullptr;     // kcs_row's P per (CTA, configuration, thread), L2-resident
  int pcache_cfg = 1;
  int ka_block = 32, kc_block = 128;
  bool all_mono = true;
  bool df = true;                 // double-float only when every plan opted in (LAM_ARITH_DOUBLE_FLOAT)
  size_t ka_smem = 0, kc_smem = 0;
  int n_sm = 1, max_ctas = 1;
  // tuning and graph
  int ctas_per_sm = 0;
  int rows_per_item = 0;
  int chunk_ctas = 0;             // CTAs per SM the instances' thickness chunks are sized for
  bool broken = false;            // tuning failed part-way: the launch tables may point at freed plan tables
  double tuned_ms[36] = {};
  std::vector<double*> inst_EG;   // per persistent instance: its mesh's Gram blocks
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double*> last_values;
};

namespace lam {

template <typename T>
static lam_status batch_upload(lam_batch& B, T** dst, const T* src, size_t n) {
  void* p = nullptr;
  const cudaError_t e = device_alloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu) failed: %s", std::max<size_t>(n, 1) * sizeof(T), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LAM_ERR_OOM : LAM_ERR_CUDA;
  }
  B.allocs.push_back(p);
  if (n) LAM_CUDA(cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice));
  *dst = static_cast<T*>(p);
  return LAM_OK;
}

static bool same_mesh(const Plan& a, const Plan& b) {
  auto same_basis = [](const Basis& x, const Basis& y) { return x.kind == y.kind && x.p == y.p && x.knots == y.knots; };
  return same_basis(a.u, b.u) && same_basis(a.v, b.v) && a.ctrl == b.ctrl && a.weights == b.weights &&
         a.nqu == b.nqu && a.nqv == b.nqv;
}

// Eq. Q arguments of one instance (pointers into the plan's device tables).
static KbArgs batch_kb_args(const Plan& P) {
  const Device& D = *P.dev;
  KbArgs a{};
  a.npairs = P.nnz_t;
  a.ncfg = (int)P.cfg_mat.size();
  a.nqt = P.nqt;
  a.q1 = P.t.p + 1;
  a.tp_row = D.tp_row;
  a.tp_col = D.tp_col;
  a.tp_e0 = D.tp_e0;
  a.tp_e1 = D.tp_e1;
  a.firstT = D.firstT;
  a.piece_begin = D.piece_begin;
  a.piece_cfg = D.piece_cfg;
  a.tabT = D.tabT;
  a.wT = D.wT;
  a.q = D.q;
  a.qdf = D.qdf;
  return a;
}

// The persistent sequence: memsets, Eq. Q, Gram blocks, double-float combine,
// exponent check, conditional FP64 combine.
constexpr int kBatchRows[3] = {1, 2, 4};  // rows per work item tried by the autotuner
constexpr int kBatchChunkCtas[3] = {4, 3, 2};  // CTAs per SM the thickness chunks are sized for (autotuner)
static lam_status batch_launch(lam_batch& B, int ctas_per_sm, int rows_index, cudaStream_t s) {
  const int n = (int)B.persistent.size();
  if (n == 0) return LAM_OK;
  LAM_CUDA(cudaMemsetAsync(B.d_flags, 0, 2 * n * sizeof(int), s));
  LAM_CUDA(cudaMemsetAsync(B.d_counter, 0, 2 * sizeof(unsigned long long), s));
  kb_batch<<<(unsigned)((B.total_pairs + 127) / 128), 128, 0, s>>>(B.d_kb, B.d_pair_prefix, n);
  LAM_CUDA(cudaGetLastError());
  if (B.df)
    ka_batch<true><<<(unsigned)B.total_elems, B.ka_block, B.ka_smem, s>>>(B.d_ka, B.d_elem_prefix, B.n_meshes);
  else
    ka_batch<false><<<(unsigned)B.total_elems, B.ka_block, B.ka_smem, s>>>(B.d_ka, B.d_elem_prefix, B.n_meshes);
  LAM_CUDA(cudaGetLastError());
  BatchKcArgs b{};
  b.kc = B.d_kc;
  b.row_prefix = B.d_row_prefix[rows_index];
  b.rows_per_item = kBatchRows[rows_index];
  b.order = B.d_order;
  b.mono = B.d_mono;
  b.n = n;
  b.counter = B.d_counter;
  b.flags = B.d_flags;
  b.pcache = B.d_pcache;
  b.pcache_cfg = B.pcache_cfg;
  const unsigned grid = (unsigned)(ctas_per_sm * B.n_sm);
  if (!B.df) {  // FP64 for every instance
    if (B.all_mono)
      kc_batch<true, false, false><<<grid, B.kc_block, B.kc_smem, s>>>(b);
    else
      kc_batch<false, false, false><<<grid, B.kc_block, B.kc_smem, s>>>(b);
    LAM_CUDA(cudaGetLastError());
    return LAM_OK;
  }
  if (B.all_mono)
    kc_batch<true, true><<<grid, B.kc_block, B.kc_smem, s>>>(b);
  else
    kc_batch<false, true><<<grid, B.kc_block, B.kc_smem, s>>>(b);
  LAM_CUDA(cudaGetLastError());
  kc_batch_check<<<(n + 127) / 128, 128, 0, s>>>(B.d_flags, n);
  LAM_CUDA(cudaGetLastError());
  b.counter = B.d_counter + 1;
  if (B.all_mono)
    kc_batch<true, false><<<grid, B.kc_block, B.kc_smem, s>>>(b);
  else
    kc_batch<false, false><<<grid, B.kc_block, B.kc_smem, s>>>(b);
  LAM_CUDA(cudaGetLastError());
  return LAM_OK;
}

// Resident combine CTAs per SM by registers (64 per thread) and by shared
// memory (dynamic + the kernel's static variables + 1 KB reserved per CTA).
static void batch_max_ctas(lam_batch& B) {
  size_t stat = 0;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kc_batch<true, false, false>) == cudaSuccess) stat = std::max(stat, fa.sharedSizeBytes);
  if (cudaFuncGetAttributes(&fa, kc_batch<false, false, false>) == cudaSuccess) stat = std::max(stat, fa.sharedSizeBytes);
  if (cudaFuncGetAttributes(&fa, kc_batch<true, true>) == cudaSuccess) stat = std::max(stat, fa.sharedSizeBytes);
  cudaGetLastError();
  const int by_regs = std::max(1, 65536 / (64 * B.kc_block));
  const int by_smem = (int)(233472 / (B.kc_smem + stat + 1024));
  B.max_ctas = std::max(1, std::min(4, std::min(by_regs, by_smem)));
}

// The combine's dynamic shared memory, for every instantiation the batch may launch.
static lam_status batch_combine_smem(lam_batch& B) {
  const int ks = (int)B.kc_smem;
  if (cudaFuncSetAttribute(kc_batch<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) != cudaSuccess ||
      cudaFuncSetAttribute(kc_batch<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) != cudaSuccess ||
      cudaFuncSetAttribute(kc_batch<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) != cudaSuccess ||
      cudaFuncSetAttribute(kc_batch<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) != cudaSuccess ||
      cudaFuncSetAttribute(kc_batch<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kc_batch<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ks) !=
          cudaSuccess) {
    cudaGetLastError();
    set_error("lam_batch: combine shared memory (%zu bytes)", B.kc_smem);
    return LAM_ERR_UNSUPPORTED;
  }
  return LAM_OK;
}

// Thickness chunks of every persistent instance sized for `ctas` CTAs per SM:
// the plans' chunks are rebuilt where their budget changes and their
// configuration tables re-uploaded (which also moves their Q buffers), then
// the instances' arguments, the combine's shared memory and its CTA limit are
// refreshed. The values move by rounding only: a chunk shares a slice between
// pairs whose Q agree up to rounding, using the Q of its first such pair.
static lam_status batch_rechunk(lam_batch& B, int ctas) {
  const int n = (int)B.persistent.size();
  std::vector<KbArgs> kb(n);
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    Plan& P = B.plans[B.persistent[k]]->p;
    const size_t before = kcs_budget(P);
    const int old = P.chunk_ctas;
    P.chunk_ctas = ctas;
    if (kcs_budget(P) != before) {
      build_chunks(P);
      if (!use_stream(P)) {  // not expected for a larger budget: keep the previous chunks
        P.chunk_ctas = old;
        build_chunks(P);
      }
      P.cfg_dirty = true;
      const lam_status st = ensure_device(P);
      if (st != LAM_OK) return st;
    }
    kb[k] = batch_kb_args(P);
    KcArgs kc = kc_args(P, nullptr);
    kc.EG = B.inst_EG[k];
    kc.values = B.h_kc[k].values;
    B.h_kc[k] = kc;
    smem = std::max(smem, kcs_smem(P));
  }
  LAM_CUDA(cudaMemcpy(B.d_kb, kb.data(), n * sizeof(KbArgs), cudaMemcpyHostToDevice));
  LAM_CUDA(cudaMemcpy(B.d_kc, B.h_kc, n * sizeof(KcArgs), cudaMemcpyHostToDevice));
  B.kc_smem = smem;
  batch_max_ctas(B);
  B.chunk_ctas = ctas;
  return batch_combine_smem(B);
}

static void batch_free(lam_batch* B) {
  if (!B) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (B->device >= 0) cudaSetDevice(B->device);
  cudaDeviceSynchronize();
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
  for (void* p : B->allocs) cudaFree(p);
  if (B->h_kc) cudaFreeHost(B->h_kc);
  if (cur >= 0) cudaSetDevice(cur);
  delete B;
}

}  // namespace lam

extern "C" {

lam_status lam_batch_create(lam_batch** out, lam_plan* const* plans, int32_t n_plans) {
  if (!out || !plans || n_plans < 1) {
    lam::set_error("lam_batch_create: NULL argument or no plans");
    return LAM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i]) {
      lam::set_error("lam_batch_create: plan %d is NULL", i);
      return LAM_ERR_INVALID_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) {
        lam::set_error("lam_batch_create: plan %d appears twice", i);
        return LAM_ERR_INVALID_ARG;
      }
  }
  lam_batch* B = new (std::nothrow) lam_batch();
  if (!B) {
    lam::set_error("lam_batch_create: out of host memory");
    return LAM_ERR_OOM;
  }
  lam_status st = LAM_OK;
#define BCHECK(x)           \
  do {                      \
    if ((st = (x)) != LAM_OK) { \
      lam::batch_free(B);   \
      return st;            \
    }                       \
  } while (0)
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    lam::set_error("lam_batch_create: no CUDA device");
    delete B;
    return LAM_ERR_CUDA;
  }
  B->device = cur;
  B->plans.assign(plans, plans + n_plans);
  for (int i = 0; i < n_plans; ++i) {
    lam::Plan& P = plans[i]->p;
    BCHECK(lam::check_limits(P));
    BCHECK(lam::ensure_device(P));
    B->df = B->df && P.arith == LAM_ARITH_DOUBLE_FLOAT;
    B->versions.push_back(P.cfg_version);
    B->nnz_total += P.nnz;
  }
  cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, cur);
  // distinct meshes and their shared Gram-block buffers
  std::vector<int> mesh_of(n_plans, -1), mesh_rep;
  for (int i = 0; i < n_plans; ++i) {
    if (plans[i]->p.shell) continue;  // general extrusions are assembled one by one (below)
    for (size_t g = 0; g < mesh_rep.size() && mesh_of[i] < 0; ++g)
      if (lam::same_mesh(plans[mesh_rep[g]]->p, plans[i]->p)) mesh_of[i] = (int)g;
    if (mesh_of[i] < 0) {
      mesh_of[i] = (int)mesh_rep.size();
      mesh_rep.push_back(i);
    }
  }
  B->n_meshes = (int)mesh_rep.size();
  std::vector<double*> mesh_EG(B->n_meshes);
  std::vector<lam::KaLocalArgs> ka(B->n_meshes);
  std::vector<int64_t> elem_prefix(B->n_meshes + 1, 0);
  for (int g = 0; g < B->n_meshes; ++g) {
    const lam::Plan& P = plans[mesh_rep[g]]->p;
    BCHECK(lam::alloc_dev(B->allocs, &mesh_EG[g], (size_t)P.u.nel * P.v.nel * 9 * lam::ka_npl(P)));
    ka[g] = lam::KaLocalArgs{};
    ka[g].ip = lam::inplane_args(P);
    ka[g].nel = P.u.nel * P.v.nel;
    ka[g].EG = mesh_EG[g];
    elem_prefix[g + 1] = elem_prefix[g] + ka[g].nel;
    B->ka_block = std::max(B->ka_block, lam::ka_block(P));
    B->ka_smem = std::max(B->ka_smem, lam::ka_smem(P));
  }
  B->total_elems = elem_prefix[B->n_meshes];
  // instances of the persistent combine, largest first
  B->inst_slot.assign(n_plans, -1);
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i]->p.shell && lam::use_stream(plans[i]->p))
      B->persistent.push_back(i);
    else
      B->fallback.push_back(i);
  }
  std::stable_sort(B->persistent.begin(), B->persistent.end(),
                   [&](int x, int y) { return plans[x]->p.nnz > plans[y]->p.nnz; });
  const int n = (int)B->persistent.size();
  std::vector<lam::KbArgs> kb(n);
  std::vector<lam::KcArgs> kc(n);
  std::vector<int64_t> pair_prefix(n + 1, 0);
  std::vector<std::vector<int64_t>> row_prefix(3, std::vector<int64_t>(n + 1, 0));
  std::vector<int> order(n), mono(n);
  for (int k = 0; k < n; ++k) {
    const int i = B->persistent[k];
    B->inst_slot[i] = k;
    lam::Plan& P = plans[i]->p;
    kb[k] = lam::batch_kb_args(P);
    pair_prefix[k + 1] = pair_prefix[k] + P.nnz_t;
    kc[k] = lam::kc_args(P, nullptr);
    kc[k].EG = mesh_EG[mesh_of[i]];
    B->inst_EG.push_back(mesh_EG[mesh_of[i]]);
    order[k] = k;
    mono[k] = P.monoclinic ? 1 : 0;
    B->all_mono = B->all_mono && P.monoclinic;
    for (int r = 0; r < 3; ++r)
      row_prefix[r][k + 1] = row_prefix[r][k] + (P.ns + lam::kBatchRows[r] - 1) / lam::kBatchRows[r];
    B->kc_block = std::max(B->kc_block, lam::kcs_block(P));
    B->kc_smem = std::max(B->kc_smem, lam::kcs_smem(P));
  }
  B->total_pairs = pair_prefix[n];
  BCHECK(lam::batch_upload(*B, &B->d_kb, kb.data(), kb.size()));
  BCHECK(lam::batch_upload(*B, &B->d_pair_prefix, pair_prefix.data(), pair_prefix.size()));
  BCHECK(lam::batch_upload(*B, &B->d_ka, ka.data(), ka.size()));
  BCHECK(lam::batch_upload(*B, &B->d_elem_prefix, elem_prefix.data(), elem_prefix.size()));
  BCHECK(lam::batch_upload(*B, &B->d_kc, kc.data(), kc.size()));
  for (int r = 0; r < 3; ++r) BCHECK(lam::batch_upload(*B, &B->d_row_prefix[r], row_prefix[r].data(), row_prefix[r].size()));
  BCHECK(lam::batch_upload(*B, &B->d_order, order.data(), order.size()));
  BCHECK(lam::batch_upload(*B, &B->d_mono, mono.data(), mono.size()));
  std::vector<int> zeros(2 * std::max(n, 1), 0);
  BCHECK(lam::batch_upload(*B, &B->d_flags, zeros.data(), zeros.size()));
  std::vector<unsigned long long> cz(2, 0ull);
  BCHECK(lam::batch_upload(*B, &B->d_counter, cz.data(), cz.size()));
  if (cudaMallocHost(reinterpret_cast<void**>(&B->h_kc), std::max(n, 1) * sizeof(lam::KcArgs)) != cudaSuccess) {
    lam::set_error("lam_batch_create: cudaMallocHost failed");
    lam::batch_free(B);
    return LAM_ERR_OOM;
  }
  std::copy(kc.begin(), kc.end(), B->h_kc);
  for (int k = 0; k < n; ++k) B->pcache_cfg = std::max(B->pcache_cfg, kc[k].ncfg);
  B->last_values.assign(n_plans, nullptr);
  lam::batch_max_ctas(*B);
  // the P cache of every CTA the combine can ever run per SM (registers bound it, whatever the chunking)
  const int pcache_ctas = std::max(1, std::min(4, 65536 / (64 * B->kc_block)));
  BCHECK(lam::alloc_dev(B->allocs, &B->d_pcache, (size_t)pcache_ctas * B->n_sm * 2 * B->pcache_cfg * B->kc_block));
  if (B->ka_smem > 48 * 1024) {
    if (cudaFuncSetAttribute(lam::ka_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->ka_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(lam::ka_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->ka_smem) !=
            cudaSuccess) {
      lam::set_error("lam_batch_create: K-a shared memory");
      lam::batch_free(B);
      return LAM_ERR_UNSUPPORTED;
    }
  }
  BCHECK(lam::batch_combine_smem(*B));
#undef BCHECK
  lam::set_error("");
  *out = B;
  return LAM_OK;
}

lam_status lam_batch_assemble(lam_batch* B, double* const* d_values, void* stream) {
  if (!B || !d_values) {
    lam::set_error("lam_batch_assemble: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  if (B->broken) {
    lam::set_error("lam_batch_assemble: an earlier call failed while tuning the batch; recreate the batch");
    return LAM_ERR_INVALID_ARG;
  }
  const int np = (int)B->plans.size();
  for (int i = 0; i < np; ++i) {
    if (!d_values[i]) {
      lam::set_error("lam_batch_assemble: values of plan %d are NULL", i);
      return LAM_ERR_INVALID_ARG;
    }
    if (B->plans[i]->p.cfg_version != B->versions[i]) {
      lam::set_error("lam_batch_assemble: plan %d was updated after the batch was created; recreate the batch", i);
      return LAM_ERR_INVALID_ARG;
    }
  }
  int cur = -1;
  LAM_CUDA(cudaGetDevice(&cur));
  if (cur != B->device) {
    lam::set_error("lam_batch_assemble: batch lives on device %d, current device is %d", B->device, cur);
    return LAM_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lam_status st;
  // value pointers of the persistent instances
  bool changed = false;
  for (int i = 0; i < np; ++i)
    if (B->inst_slot[i] >= 0 && B->last_values[i] != d_values[i]) changed = true;
  const int n = (int)B->persistent.size();
  if (changed && n > 0) {
    // the pinned staging copy must not be rewritten while an earlier upload from it may be pending
    LAM_CUDA(cudaDeviceSynchronize());
    for (int i = 0; i < np; ++i)
      if (B->inst_slot[i] >= 0) {
        B->h_kc[B->inst_slot[i]].values = d_values[i];
        B->last_values[i] = d_values[i];
      }
    LAM_CUDA(cudaMemcpyAsync(B->d_kc, B->h_kc, n * sizeof(lam::KcArgs), cudaMemcpyHostToDevice, s));
  }
  if (n > 0 && B->ctas_per_sm == 0) {
    // autotune: one full sequence per candidate (thickness-chunk depth x rows
    // per work item x CTAs per SM that the chunks leave room for), after a
    // warm-up per chunk depth
    cudaEvent_t e0, e1;
    LAM_CUDA(cudaEventCreate(&e0));
    LAM_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int best_h = 0, best_r = 0, best_c = 1;
    for (int h = 0; h < 3; ++h) {
      if ((st = lam::batch_rechunk(*B, lam::kBatchChunkCtas[h])) != LAM_OK) {
        B->broken = true;
        return st;
      }
      if ((st = lam::batch_launch(*B, B->max_ctas, 0, s)) != LAM_OK) return st;
      for (int r = 0; r < 3; ++r)
        for (int c = 1; c <= B->max_ctas; ++c) {
          LAM_CUDA(cudaEventRecord(e0, s));
          if ((st = lam::batch_launch(*B, c, r, s)) != LAM_OK) return st;
          LAM_CUDA(cudaEventRecord(e1, s));
          LAM_CUDA(cudaEventSynchronize(e1));
          float ms = 0.0f;
          LAM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          B->tuned_ms[(h * 3 + r) * 4 + c - 1] = ms;
          if (ms < best) {
            best = ms;
            best_h = h;
            best_r = r;
            best_c = c;
          }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (lam::kBatchChunkCtas[best_h] != B->chunk_ctas &&
        (st = lam::batch_rechunk(*B, lam::kBatchChunkCtas[best_h])) != LAM_OK) {
      B->broken = true;
      return st;
    }
    B->ctas_per_sm = best_c;
    B->rows_per_item = lam::kBatchRows[best_r];
    // capture the tuned sequence on a stream of the batch's own
    LAM_CUDA(cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    LAM_CUDA(cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal));
    st = lam::batch_launch(*B, B->ctas_per_sm, best_r, B->capture_stream);
    cudaError_t ce = cudaStreamEndCapture(B->capture_stream, &graph);
    if (st != LAM_OK) return st;
    if (ce != cudaSuccess) {
      lam::set_error("lam_batch_assemble: graph capture failed: %s", cudaGetErrorString(ce));
      return LAM_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      B->exec = nullptr;
      lam::set_error("lam_batch_assemble: graph instantiation failed: %s", cudaGetErrorString(ce));
      return LAM_ERR_CUDA;
    }
  }
  // the values of this call come from the tuned sequence (the last candidate the
  // autotuner timed may have used another chunk depth, which moves their rounding)
  if (n > 0) LAM_CUDA(cudaGraphLaunch(B->exec, s));
  for (int i : B->fallback)
    if ((st = lam_assemble_split(B->plans[i], d_values[i], stream)) != LAM_OK) return st;
  return LAM_OK;
}

lam_status lam_batch_get_info(const lam_batch* B, lam_batch_info* info) {
  if (!B || !info) {
    lam::set_error("lam_batch_get_info: NULL argument");
    return LAM_ERR_INVALID_ARG;
  }
  *info = lam_batch_info{};
  info->n_plans = (int32_t)B->plans.size();
  info->n_meshes = B->n_meshes;
  info->nnz_total = B->nnz_total;
  info->n_persistent = (int32_t)B->persistent.size();
  info->ctas_per_sm = B->ctas_per_sm;
  info->graph = B->exec ? 1 : 0;
  info->rows_per_item = B->rows_per_item;
  info->chunk_ctas = B->chunk_ctas;
  for (int k = 0; k < 36; ++k) info->tuned_ms[k] = B->tuned_ms[k];
  return LAM_OK;
}

lam_status lam_batch_destroy(lam_batch* B) {
  lam::batch_free(B);
  return LAM_OK;
}

}  // extern "C"
