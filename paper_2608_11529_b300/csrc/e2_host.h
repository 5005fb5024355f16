// Host-side internals shared by the C-ABI translation units (plan,
// execution, batches, gradient, reference solver): the plan structures, the
// workspace layout and the stream-ordered launch helpers.  Not installed.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "e2_common.cuh"
#include "e2_kernels.cuh"

namespace e2 {

using Pat = std::array<int, E2_MAX_DAS>;

int64_t binom_h(int n, int k);

struct HostList {
  int count = 0;
  std::vector<Pat> pats;
  std::vector<int64_t> patoff;
  int64_t n = 0;
  std::vector<int64_t> key2off;
  size_t o_str = 0, o_key = 0, o_patoff = 0, o_patocc = 0, o_eA = 0, o_U = 0;
  bool df = false;               // float-float copies of e_A and U (a class on the sliced path uses the list)
  size_t o_eAdf = 0, o_Udf = 0;
};

// Column tiles of a dense class with a compacted contraction (see ColTiles).
struct ColPlan {
  bool built = false;
  std::vector<int32_t> perm;   // [tiles * 64] list index, -1 = padding
  std::vector<int32_t> tdesc;  // [tiles][4] {koff, klen, ktrue, 0}
  std::vector<int32_t> klist;  // [krows]
  std::vector<int32_t> pos;    // [tiles][Kp] compacted row of table row x in tile j, -1 if absent
  int64_t tiles = 0, krows = 0;
  int maxklen = 0;             // longest compacted contraction of a tile
  int gran = 8;                // contraction granularity of the tiles (4: a k = 4 tail step)
  int pbn = 80;                // width of the backward's compacted product tiles (32, 48, 64 or 80)
  int64_t gd_ctas = 0;         // sum over tiles of ceil(klen / pbn)
  double ratio = 1.0;          // krows / (tiles * Kp): share of the dense contraction
  size_t o_perm = 0, o_tdesc = 0, o_klist = 0, o_pos = 0, o_Dc = 0;  // o_Dc: per-root D region
};

// Bump allocator over the workspace (256-byte aligned segments).
struct Layout {
  size_t top = 0;
  size_t take(size_t bytes) {
    size_t o = top;
    top += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace e2

struct e2_problem {
  e2_desc d;
  std::vector<uint8_t> frozen;
  int das_size[E2_MAX_DAS], das_min[E2_MAX_DAS], das_max[E2_MAX_DAS];
  int n, nocc, ncc, nvc, nx, na, N;
  std::vector<int32_t> cc, vc;
  e2::DevDas das;
  int nkeys;
  std::vector<e2::Pat> ppats;          // P patterns (address order)
  std::vector<e2::HostList> lists;     // unique string lists
  int list_of[E2_NCLASS];          // class -> list (-1: no strings)
  int listP;
  // integral / table shapes
  int ntp;
  int64_t nvp, ncp;
  int64_t M[E2_NCLASS];            // rows of each class
  int Kp[E2_NCLASS];               // padded contraction length of the dense classes
  int KpT, KpTU, Kp11;             // rows of the D^t / D^tu / D^{t+u} tables
  double q_per_class[E2_NCLASS];
  // workspace layout
  size_t ws_bytes;
  size_t o_plan, plan_bytes;
  size_t o_binom, o_EO, o_E0p, o_E0, o_G, o_epsh, o_dg, o_wt, o_Bo, o_f, o_cc, o_vc;
  size_t o_status;  // device status word: flags + smallest |D| key per (root, class)
  size_t o_xc, o_xv;  // external subspace ids of one-hole / one-particle subspaces (plan region)
  std::vector<int32_t> xc, xv;  // their host copies (-1: no limit below two)
  bool ext_das = false;         // some external subspace limit is one
  double q_full[E2_NCLASS];     // class sizes without external subspace limits
  int shard_rank = 0, shard_n = 1;  // e2_set_shard: this rank's share of every class's units
  size_t o_rows[E2_NCLASS], o_W[E2_NCLASS];
  size_t o_G22, o_X01, o_X10, o_X00;
  size_t o_vaY, o_vaZ, o_vaX, va_cap;
  size_t o_xYc, o_xZaa, o_x12, o_x01;
  size_t o_DT, o_DTD, o_DTU, o_DTDUD, o_DTDU;  // per-root stride below
  size_t d_stride;                              // bytes of one root's D tables
  bool multi_slot = false;                      // set while a batch uses the job: a table slot per root
  int slots = 0;                                // with multi_slot: slots in use (root r in slot r % slots; 0 = n_roots)
  size_t o_g1, o_g2, g_stride;                  // gram outputs per root
  size_t o_part, o_partoff, o_partcnt, o_e2c;
  int64_t part_cnt[E2_NCLASS];
  std::vector<int64_t> part_off;                // [n_roots][E2_NCLASS]
  std::vector<unsigned char> plan_blob;         // host image of the plan region
  // launch shapes of the sparse / elementwise classes
  int nvb;
  // optional CUDA events around each class kernel of root 0 (bench hooks)
  cudaEvent_t prof[2 * E2_NCLASS];
  bool prof_on = false;
  int64_t launches = 0;  // kernels enqueued by the last e2_forward
  // reference solver region
  int sv_mmax;
  size_t o_sV, o_sS, o_sX, o_sR, o_sD, o_sT, o_sG, o_sY, solve_bytes;
  // adjoint region
  size_t o_dstart;                   // first D table of the root-0 slot
  int64_t chunk_rows[E2_NCLASS] = {};  // dense-class rows per adjoint chunk
  int64_t chunk_rows_plan[E2_NCLASS] = {};  // the planned (largest) values of the two chunk sizes
  int z22_chunk = 1, z22_plan = 1;   // core pairs per chunk of the (2,2) adjoint
  size_t o_gD, o_bT, o_bHrow, o_bHcol, o_bScalT, o_bHsum, o_bHA, o_bRowdot;
  size_t o_bGT, o_bGH, o_bGV, o_bC22p, o_bH22p, o_bV22, o_bC22, o_bGc, o_bSig, o_bGf, o_bNx, o_bNt, o_bNd, o_bScal;
  // factor gradient
  int64_t npair;
  size_t o_bGW[E2_NCLASS], o_bHm, o_bHocc, o_bZ, o_bGe, o_bGea, o_bNtt, o_bGG, o_bGt, o_bGh, o_bTsh;
  size_t o_bGX01, o_bGX10, o_bGX00, o_bHs22, o_bP22, o_bG22c, o_bGg22, o_bCs, o_bGB, o_bFtr, o_bGw;
  size_t o_bPart, bpart_bytes;  // split-K segments
  size_t tsh_bytes;
  size_t o_bGDc, o_bGWc, gwc_bytes;
  size_t bwd_bytes;
  // compacted column tiles of the dense classes and whether each class uses them
  e2::ColPlan cplan[E2_NCLASS];
  bool use_cols[E2_NCLASS] = {};
  // sliced bf16 contraction of the dense classes (real length 2 Kp <= 256):
  // W slices and row exponents beside W, D slices and string exponents in
  // each root's table slot
  bool oz_ok[E2_NCLASS] = {};        // planned (buffers laid out)
  bool use_oz[E2_NCLASS] = {};       // in use
  int oz_kq[E2_NCLASS] = {};
  int64_t oz_mpad[E2_NCLASS] = {}, oz_npad[E2_NCLASS] = {};
  bool use_oz_setup = false;         // the setup's integral products on the sliced GEMM
  size_t o_ozS = 0, ozS_bytes = 0;   // their scratch (over the region the D tables take later)
  bool use_oz_adj = false;           // the adjoint's Gamma products and Cs on the sliced GEMM
  size_t o_bOz = 0, bOz_bytes = 0;   // their scratch (backward region)
  size_t o_bC2 = 0;                  // |c_A|^2 / n of the class-(2,2) strings, float-float (backward)
  size_t o_ozA[E2_NCLASS] = {}, o_ozRx[E2_NCLASS] = {}, o_ozB[E2_NCLASS] = {}, o_ozCx[E2_NCLASS] = {};
};

struct e2_batch {
  std::vector<e2_problem*> jobs;
  std::vector<size_t> off;          // workspace offset of each job's forward layout
  std::vector<size_t> o_c;          // per job: device copy of its reference coefficients (all roots)
  size_t o_jobs = 0, o_sjobs = 0, o_segs = 0, o_counter = 0, bytes = 0;  // o_counter: one per launch
  std::vector<e2::GemmJob> gj;      // absolute pointers, built by e2_batch_prepare
  std::vector<e2::SparseJob> sj;
  std::vector<e2::WorkSeg> segs;      // runs of every launch, launch after launch
  std::vector<int64_t> seg0, nseg, items;  // per launch: first run, runs, items
  int64_t n_items = 0;
  int64_t max_gj = 0, max_sj = 0, max_segs = 0;
  int roots_per_launch = 0;           // 0: every root of every job in one launch
  int n_launch = 1;                   // persistent launches (root groups)
  const void* prepared = nullptr;
  int64_t launches = 0;
};

namespace e2 {

// ---- planning (e2_plan.cu)
e2_status build_plan(e2_problem* P);

// ---- launch helpers (e2_api.cu)
inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }
// threads and dynamic shared memory of k_class22_rows's per-row occupation
// sums (one column of na doubles per thread, at most 40 KiB, under the
// 48 KiB a block may take without opting in)
inline int occ_threads(int na) { return na <= 20 ? 256 : na <= 40 ? 128 : 64; }
inline size_t occ_smem(int na) { return (size_t)na * occ_threads(na) * sizeof(double); }

// kernels enqueued by the current host thread (read back as the count of one call)
extern thread_local int64_t g_launches;
// scratch for split-K segments of the GEMM helpers (set while a pass that
// owns such a region runs; null: no split)
extern thread_local void* g_splitk;
extern thread_local size_t g_splitk_bytes;

struct Ctx {
  const int64_t* binom;
  double *G, *epsh, *EO, *E0p, *E0d, *dg, *wt;
  double2 *Bo, *f;
  DevSpace sp;
};

struct Tabs {
  double2 *DT, *DTD, *DTU, *DTDUD, *DTDU;
};

DevList dev_list(const e2_problem* P, int li, unsigned char* ws);
Ctx ctx(const e2_problem* P, unsigned char* ws);
unsigned char* slot_base(const e2_problem* P, unsigned char* ws, int r);
Tabs tables(const e2_problem* P, unsigned char* ws, int r);
ColTiles col_tiles(const e2_problem* P, unsigned char* ws, int r, int cls);
// the status word (flags, then the smallest |D| key per root and class) and its slots
// Partial slots of all roots and classes (contiguous from o_part).
inline int64_t part_total(const e2_problem* P) {
  int64_t t = 0;
  for (int c = 0; c < E2_NCLASS; ++c) t += P->part_cnt[c];
  return t * P->d.n_roots;
}

// Units of class cls that the forward can split across ranks: row tiles of a
// dense class, (core pair, virtual block pair) units of (2,2), rows (virtual
// a or core i) of (0,1) and (1,0), 256-string blocks of (0,0).
inline int64_t shard_units(const e2_problem* P, int cls) {
  if (P->part_cnt[cls] == 0) return 0;
  switch (cls) {
    case 2: case 4: case 5: case 6: case 7: return (P->M[cls] + 63) / 64;
    case 8: return P->ncp * ((int64_t)P->nvb * (P->nvb + 1) / 2);
    case 1: return P->nvc;
    case 3: return P->ncc;
    default: return (P->lists[P->list_of[0]].n + 255) / 256;
  }
}
// This rank's contiguous share [u0, u1) of them (all of them without shards).
inline void shard_range(const e2_problem* P, int cls, int64_t& u0, int64_t& u1) {
  const int64_t n = shard_units(P, cls);
  u0 = n * P->shard_rank / P->shard_n;
  u1 = n * (P->shard_rank + 1) / P->shard_n;
}

// the device address of e2_forward_noalloc's static scratch on the current device (null on failure)
void* noalloc_scratch();
inline unsigned long long* status_word(const e2_problem* P, unsigned char* ws) {
  return (unsigned long long*)(ws + P->o_status);
}
inline unsigned long long* dmin_slot(const e2_problem* P, unsigned char* ws, int r, int cls) {
  return status_word(P, ws) + 1 + (int64_t)r * E2_NCLASS + cls;
}
// operands of the sliced contraction of class cls for root r
OzOperands oz_operands(const e2_problem* P, unsigned char* ws, int r, int cls);
// the sliced contraction with its Epstein-Nesbet epilogue; partial: one slot
// per 64 x 64 tile, [column tile][row tile] (e2_ozaki.cu)
// (row tiles tm0 .. tm0 + ntm - 1; ntm < 0: to the last)
void launch_class_oz(cudaStream_t st, int cls, const OzOperands& op, int64_t M, int64_t N, const RowInfo* rows,
                     const double* E0p, double b, double* partial, unsigned long long* dmin, int64_t tm0 = 0,
                     int64_t ntm = -1);
// class (2,2) in float-float (e2_ozaki.cu), the partials of k_class22
void launch_class22_df(cudaStream_t st, const DevList& L, const DevSpace& sp, const float2* eAdf, const float2* Udf,
                       const double2* c, const double* g2, const double* epsh, const double* G, const double* E0p,
                       double b, int nvb, int64_t ncp, double* partial, unsigned long long* dmin, int64_t u0 = 0,
                       int64_t u1 = -1);
// float-float forms of per-row adjoint sums (e2_ozaki.cu): occupation sums of
// eta given as float-float pairs, and the per-row sums of class (2,2)
void launch_hocc_df(cudaStream_t st, const float2* H, const DevList& L, int na, int64_t rows, double* Hocc);
void launch_class22_rows_df(cudaStream_t st, const DevList& L, const DevSpace& sp, const float2* eAdf,
                            const float2* Udf, const float2* c2df, const double* g2, const double* epsh,
                            const double* G, const double* E0p, double b, double s, int64_t rows, double* hsum,
                            double* Hocc, double* P22);
// its adjoint mode over one row chunk of the backward pass (see AdjOut)
void launch_class_oz_adj(cudaStream_t st, int cls, const OzOperands& op, int64_t M, int64_t N, const RowInfo* rows,
                         const double* E0p, double b, const AdjOut& adj);
// C (+)= A B (complex, strided as zgemm) through exact bf16 slices (4 or 5 per
// operand) with float-float accumulation (e2_ozaki.cu); lower >= 0: only tiles reaching
// n <= lower + m.  Needs zgemm_sliced_bytes(M, max(N, Nslice), K) of scratch
// (returns false, launching nothing, when it is short).  B is sliced over
// Nslice >= N columns when given, so that reuse_b can keep those slices for
// a following call on the same scratch and B with a narrower N.  a_df: A holds
// float-float quadruples (re.hi, re.lo, im.hi, im.lo) instead of FP64 pairs.
size_t zgemm_sliced_bytes(int64_t M, int64_t N, int64_t K, int slices = OZ_S);
bool zgemm_sliced(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak,
                  int conjA, const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm,
                  int64_t csn, int beta, int64_t lower, unsigned char* scratch, size_t scratch_bytes,
                  int64_t Nslice = 0, bool reuse_b = false, int slices = OZ_S, bool a_df = false);
// slices of the dense classes' operands (OZ_S slices): W's rows, a D table's strings
void launch_slice_rows(cudaStream_t st, const double2* A, int64_t sam, int64_t sak, int64_t M, int K, int Kq,
                       int64_t Mpad, __nv_bfloat16* out, int* rexp);
void launch_slice_cols(cudaStream_t st, const double2* B, int64_t sbk, int64_t sbn, int K, int64_t N, int Kq,
                       int64_t Npad, __nv_bfloat16* out, int* cexp);
void build_tables(const e2_problem* P, unsigned char* ws, cudaStream_t st, const double2* c, const Tabs& T, bool all);
int splitk_segments(int64_t tiles, int64_t K, size_t seg_bytes);
void dgemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double* A, int64_t sam, int64_t sak,
           const double* B, int64_t sbk, int64_t sbn, double* C, int64_t ldc, int beta);
void zgemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
           const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn, int beta,
           int bn = 64);
e2_status setup_common(e2_problem* P, const e2_inputs* in, unsigned char* ws, cudaStream_t st, bool upload = true);
void setup_classes(e2_problem* P, unsigned char* ws, cudaStream_t st);
void zgemm_gd_tiles(cudaStream_t st, const ColPlan& cp, const ColTiles& ctl, const double2* W, int Kp,
                    const double2* T, int64_t N, int64_t Mc, double2* GDc, int beta, int conjT = 1,
                    int64_t t_ld = 0);
void prepare_root(e2_problem* P, unsigned char* ws, cudaStream_t st, const double2* c, int r);
void launch_reduce(e2_problem* P, unsigned char* ws, cudaStream_t st, double* E2, double* E2_class, double* E0);

// Classes (2,2), (0,1), (1,0), (0,0) of root r (their partial slots).
template <class Mark>
void launch_sparse_classes(e2_problem* P, unsigned char* ws, cudaStream_t st, int r, const double2* c, Mark mark) {
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, r);
  DevList Lc[E2_NCLASS];
  for (int k = 0; k < E2_NCLASS; ++k) Lc[k] = dev_list(P, P->list_of[k], ws);
  const double b = P->d.level_shift_b;
  double* part = (double*)(ws + P->o_part);
  auto poff = [&](int cls) { return part + P->part_off[r * E2_NCLASS + cls]; };
  int64_t u0, u1;
  shard_range(P, 8, u0, u1);
  if (u1 > u0) {
    const DevList& L = Lc[8];
    mark(8, 0);
    if (P->use_oz[8]) {  // float-float
      const HostList& H8 = P->lists[P->list_of[8]];
      launch_class22_df(st, L, X.sp, (const float2*)(ws + H8.o_eAdf), (const float2*)(ws + H8.o_Udf), c,
                        (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b, P->nvb, P->ncp, poff(8),
                        dmin_slot(P, ws, r, 8), u0, u1);
    } else {
      // grid y: at most 65535 units per launch
      for (int64_t a = u0; a < u1; a += 65535) {
        dim3 grid(blocks(L.n), (unsigned)std::min<int64_t>(65535, u1 - a));
        (k_class22<<<grid, 256, 0, st>>>(L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b,
                                        P->nvb, poff(8), dmin_slot(P, ws, r, 8), a), ++g_launches);
      }
    }
    mark(8, 1);
  }
  shard_range(P, 1, u0, u1);
  if (u1 > u0) {
    dim3 grid(blocks(Lc[1].n), (unsigned)(u1 - u0));
    mark(1, 0);
    (k_class01<<<grid, 256, 0, st>>>(Lc[1], Lc[5], Lc[2], P->das, X.sp, X.binom, T.DT, T.DTU,
                                    (const double2*)(ws + P->o_X01), X.f, X.epsh, X.E0p + r, b, poff(1),
                                    dmin_slot(P, ws, r, 1), nullptr, nullptr, u0), ++g_launches);
    mark(1, 1);
  }
  shard_range(P, 3, u0, u1);
  if (u1 > u0) {
    dim3 grid(blocks(Lc[3].n), (unsigned)(u1 - u0));
    mark(3, 0);
    (k_class10<<<grid, 256, 0, st>>>(Lc[3], Lc[7], Lc[5], P->das, X.sp, X.binom, T.DTD, T.DT,
                                    (const double2*)(ws + P->o_X10), X.f, X.epsh, X.E0p + r, b, poff(3),
                                    dmin_slot(P, ws, r, 3), nullptr, nullptr, u0), ++g_launches);
    mark(3, 1);
  }
  shard_range(P, 0, u0, u1);
  if (u1 > u0) {
    mark(0, 0);
    (k_class00<<<(unsigned)(u1 - u0), 256, 0, st>>>(Lc[0], Lc[4], Lc[2], P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                                   (const double2*)(ws + P->o_X00), X.f, X.E0p + r, b, poff(0),
                                                   dmin_slot(P, ws, r, 0), nullptr, nullptr, u0), ++g_launches);
    mark(0, 1);
  }
}

}  // namespace e2
