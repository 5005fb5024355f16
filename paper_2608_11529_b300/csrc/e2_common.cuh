// Internal declarations shared by the host plan and the sm_103a kernels.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "e2.h"

namespace e2 {

constexpr int kMaxPat = 1024;      // occupation patterns per string list
constexpr int kMaxKeys = 1 << 20;  // size of the pattern-key table
constexpr int kBinomN = 65;        // binomial table is [65][65]
constexpr int OZ_S = 5;            // slices per operand of the sliced bf16 contraction
constexpr int OZ_ADJ_S = 4;        // slices of the adjoint's products (gradients: 2^-33 of the scales)
// Slice exponent of a row or column that holds a NaN or an infinity: the
// slices are then zero and the scale 2^(rexp + cexp) becomes NaN / infinite,
// so the product and every energy formed from it are not finite.
constexpr int OZ_NONFINITE = 1 << 20;
// Device status word (workspace, see e2_query_status): flag bits, then the
// smallest |D| per (root, class) as ordered integer keys.
constexpr unsigned long long ST_NONFINITE = 1ULL, ST_INTRUDER = 2ULL;
constexpr double kIntruderD = 1e-12;  // |D| below this with b = 0: an intruder state (Sec. 2.6)

// Operands of the sliced (bf16) dense-class contraction: row slices of W
// [OZ_S][Mpad][Kq] with one exponent per row, string slices of D
// [OZ_S][2 Npad][Kq] with one exponent per string (Kq: the real contraction
// length 2K padded to a multiple of 32), and float-float copies (hi, lo) of
// the class list's e_A [n] and U [nx + 1][n].
struct OzOperands {
  const __nv_bfloat16* A;
  int64_t Mpad;
  const int* rexp;
  const __nv_bfloat16* B;
  int64_t Npad;
  const int* cexp;
  int Kq;
  const float2* Udf;
  const float2* eAdf;
  int nx;  // U row index of an absent spinor (a zero row)
};

// Active-space partition as the kernels see it.
struct DevDas {
  int n_das;
  int n_act;
  int off[E2_MAX_DAS];     // first active-local index of each subspace
  int size[E2_MAX_DAS];
  int keymul[E2_MAX_DAS];  // pattern key = sum_s n_s * keymul[s]
};

// One list of active strings (a union of occupation-pattern blocks).
struct DevList {
  int count;                // electrons per string
  int npat;
  int64_t n;                // strings
  uint64_t* str;            // [n] active-local bitsets, in list order
  const int64_t* key2off;   // [nkeys] block offset of a pattern, -1 if absent
  const int64_t* patoff;    // [npat]
  const int32_t* patocc;    // [npat][E2_MAX_DAS]
  double* eA;               // [n]   sum_t eps^_t + 1/2 sum_{t!=u} G_tu over the string
  double* U;                // [nx+1][n]  U[x][A] = sum_{t in A} G_{X(x),t}; row nx is zero
};

// Per external row of the dense classes: U-row indices of the two
// particles (s1, s2) and two holes (i1, i2), nx when absent, and chi(e).
struct RowInfo {
  int32_t s1, s2, i1, i2;
  double chi;
};

// Adjoint outputs of the dense-class kernel (T == nullptr: forward mode).
// Rows [m_base, m_base + Mc) are processed; T holds t = s (2/n) (df/dv) V
// for those rows, Hrow[row][column tile] and Hcol[row tile][column] the
// per-tile sums of s df/dD, scal[2 * tile] = (sum s df/dD, sum s (df/dv) v);
// n = <c|c> is read from g1[0].  With part set, each tile also writes the
// forward's partial of sum f (slot tile_n * rt + global row tile), so that the
// backward pass returns E2 as well.
struct AdjOut {
  double2* T;
  double* Hm;      // optional: s df/dD per element of the chunk (same layout as T)
  double* Hrow;    // [Mc][column tiles]: per-tile row sums of eta, rows local to the chunk
  double* Hcol;    // [row tiles of the chunk][N]: per-tile column sums of eta
  double* scal;    // [row tiles of the chunk][column tiles][2]: the two per-tile scalars
  int64_t m_base, Mc;
  double s;
  const double2* g1;
  double* part;
  int64_t rt;
  int t_df;  // sliced adjoint only: T as float-float quadruples (its consumers slice them)
  // FP64 adjoint of a column-tiled class: T and Hm in tile column order,
  // element (row, tile j, column c) at [row - m_base][64 j + c] (row stride
  // t_ld = 64 x tiles; padding columns hold 0), so that the tile products
  // read contiguous row segments; otherwise [row - m_base][string] (stride N)
  int t_tile;
  int64_t t_ld;
  // forward mode only (T == nullptr): when set, the tile also writes each
  // coupling's V and D at [local row][local column] (64 x 64), for a
  // per-coupling check of one tile
  double2* probeV;
  double* probeD;
};

// Column tiles of a dense class with a compacted contraction.  The coupling
// table D [Kp][N] has structural zeros (D^{tu}_A = 0 when t or u is in A,
// and so on); the class's strings are grouped into 64-column tiles whose
// strings share occupied (or empty) spinors, and each tile contracts only
// over the rows of D that are non-zero somewhere in it:
//   perm[64 j + c]   list index of column c of tile j, -1 for padding
//   tdesc[j]         {koff, klen (multiple of 8), ktrue, 0}
//   klist[koff + k]  D row of compacted row k (0 beyond ktrue)
//   Dc[(koff + k) * 64 + c] = D[klist[koff + k]][perm[64 j + c]] (0 beyond ktrue)
// perm == nullptr: plain consecutive columns over the full Kp.
struct ColTiles {
  const int32_t* perm;
  const int4* tdesc;
  const int32_t* klist;
  const double2* Dc;
};

// One dense-class contraction of a batch (absolute device pointers).
struct GemmJob {
  const double2* W;
  const double2* D;
  int64_t M, N;
  int Kp;
  const RowInfo* rows;
  const double* U;
  const double* eA;
  const double* E0p;
  double b;
  double* partial;
  ColTiles ct;
  unsigned long long* dmin;  // smallest |D| key of the class and root (status word)
};


enum IntMode : int {
  INT_W02 = 0,  // <ab||tu>          rows (a<b), cols (t<u)
  INT_W12,      // <ab||it>          rows (i, a<b), cols t
  INT_W21,      // <at||ij>          rows (i<j, a), cols t
  INT_W11,      // f_ai | <at||iu>   rows (i, a), cols 0 | 1 + t*na + u
  INT_W20,      // <tu||ij>          rows (i<j), cols (t<u)
  INT_G22,      // |<ab||ij>|^2      rows (i<j), cols (a<b), real
  INT_X01,      // <au||vw>          rows a, cols u*ntp + (v<w)
  INT_X10,      // <tu||iv>          rows i, cols (t<u)*na + v
  INT_X00,      // <tu||vw>          rows (t<u), cols (v<w)
  INT_G22C      // <ab||ij>          rows (i<j), cols (a<b), complex
};

enum DFamily : int {
  FAM_T = 0,  // <A| a_t |Psi>
  FAM_TD,     // <A| a+_t |Psi>
  FAM_TU,     // <A| a_u a_t |Psi>, t<u
  FAM_TDUD,   // <A| a+_t a+_u |Psi>, t<u
  FAM_TDU     // row 0: c_A (A in P); row 1+t*na+u: <A| a+_t a_u |Psi>
};

// Spinor index sets used by the kernels.
struct DevSpace {
  int n, n_core, n_act, n_virt, n_occ, a0, v0;
  int ncc, nvc, nx;        // correlated core / virtual counts, nx = ncc + nvc
  const int32_t* cc;       // [ncc] global index of correlated core spinors
  const int32_t* vc;       // [nvc] global index of correlated virtual spinors
  // external subspace limits (e2_set_external_das): per correlated core /
  // virtual spinor, its subspace id when that subspace admits one hole /
  // particle only, else -1
  const int32_t* xc;       // [ncc]
  const int32_t* xv;       // [nvc]
};

// One (job, root) of a batch's element-wise classes: (2,2) and the gather
// classes (0,1), (1,0), (0,0) (absolute device pointers).  L<c> is the string
// list of class c; part / dmin hold the partial slots and smallest-|D| slots
// of classes (2,2), (0,1), (1,0), (0,0) in that order.
struct SparseJob {
  DevList L8, L1, L3, L0, L2, L4, L5, L7;
  DevDas das;
  DevSpace sp;
  const int64_t* binom;
  const double2 *c, *DT, *DTU, *DTD, *DTDU, *X01, *X10, *X00, *f;
  const double *g2, *epsh, *G, *E0p;
  double b;
  int nvb;
  double* part[4];
  unsigned long long* dmin[4];
};

// A run of work items of one kind in the persistent batch launch: items
// [first, first + count), item k of the run being tile (k / gx, k % gx) of a
// dense class (GemmJob job), or block (row or unit k / gx, string tile
// k % gx) of an element-wise class (SparseJob job; (0,0): block k).
enum WorkKind : int { WORK_TILE = 0, WORK_C22 = 1, WORK_C01 = 2, WORK_C10 = 3, WORK_C00 = 4 };
struct WorkSeg {
  int kind, job;
  int64_t first, count, gx;
};

// chi of an external row that the external subspace limits exclude: its W
// row (or |<ab||ij>|^2) is zeroed, so V = 0, and D = E0' - chi is far from 0
// and from every real denominator (|D| < 1e4 Eh), so it never reaches the
// smallest-|D| diagnostics; the denominator histogram skips it.
constexpr double kExcludedChi = -1e8;

__host__ __device__ inline int64_t pairs(int64_t n) { return n * (n - 1) / 2; }

}  // namespace e2
