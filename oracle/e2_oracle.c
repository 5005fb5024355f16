/*
 * e2_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow CPU evaluation of the Epstein-Nesbet second-order energy of a
 * multiconfigurational reference, written from the paper's definitions:
 *
 *   E2_m = sum_{K in Q} |<K|H|Psi_m>|^2 / (E0_m - H_KK)            (Eq. pt2, Eq. pt2en)
 *   H0   = P H P + diag(Q H Q)  (Epstein-Nesbet partitioning)      (Eq. zeroh)
 *   Q    = all determinants outside P that are single or double
 *          substitutions of some P determinant                     (Sec. 2.3)
 *   P    = active-space determinants of the allowed DAS occupation
 *          patterns, core full, virtuals empty                      (Sec. 2.4, Eq. DASK)
 *   frozen core / frozen virtual spinors never take part in a
 *   substitution (frozen core always occupied)                     (Sec. 2.5)
 *   imaginary level shift (E0-H_KK+i b/(E0-H_KK))^{-1}, real part (Sec. 2.6)
 *
 * Nothing here is shared with the GPU library.  Only tests, the smoke check
 * and the CPU baseline leg of the benchmark may load this file's library.
 *
 * Determinants are multi-word bitsets over all spinors; a determinant is the
 * product of creators in ascending spinor order acting on the vacuum, so
 * a_p acting on it carries (-1)^(number of occupied spinors below p).
 * Matrix elements follow the Slater-Condon rules for 0, 1 or 2 differences,
 * with H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r,
 * <pq||rs> = (pr|qs) - (ps|qr), (pq|rs) = sum_L w_L B^L_pq B^L_rs.
 * V_K is an explicit Q H P row: the sum over every P determinant within two
 * substitutions of K.
 *
 * Address of a P determinant (the order of the reference coefficients c):
 * patterns (n_1..n_k) in lexicographic order (n_1 most significant), a block
 * per pattern; inside a block, sum_s rank_s * stride_s with rank_s the colex
 * rank of the subspace-s substring (local indices, rank = sum_j C(t_j, j+1)),
 * stride_1 = 1 and stride_{s+1} = stride_s * C(size_s, n_s).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXW 20      /* up to 1280 spinors */
#define MAXDAS 8
#define MAXPAT 4096
#define NCLASS 9     /* class id = 3*holes + particles */

typedef struct { uint64_t w[MAXW]; } det_t;
typedef double complex cplx;

typedef struct {
  int n_core, n_act, n_virt, n_elec;
  int n_das;
  const int* das_size;
  const int* das_min;
  const int* das_max;
  const unsigned char* frozen;
  const double* h;      /* complex interleaved [n][n] */
  int L;
  const double* B;      /* complex interleaved [L][n][n] */
  const double* w;      /* [L] */
  double level_shift_b;
  int use_eri_cache;
  int n_threads;
} oracle_desc;

typedef struct {
  int n, n_core, n_act, n_virt, n_elec, a0, v0;
  int n_das, das_size[MAXDAS], das_min[MAXDAS], das_max[MAXDAS], das_off[MAXDAS];
  unsigned char* frozen;
  cplx* h;
  int L;
  const cplx* B;
  double* w;
  cplx* eri;          /* (pq|rs) cache, or NULL */
  double* G;          /* <pq||pq> */
  int n_pat;
  int pat[MAXPAT][MAXDAS];
  int64_t pat_off[MAXPAT + 1];
  int n_roots;
  cplx* c;            /* [n_roots][n_p] */
  double b;
  int n_threads;
  int ncc, nvc;       /* correlated core / virtual counts */
  int* corr_core;
  int* corr_virt;
  uint64_t* pstr;     /* active string of each P address */
  /* DAS subspaces of the core and virtual spaces (Sec. 2.4, Fig. 1) with
     per-subspace limits on holes / particles; xsub[p] = subspace of spinor p
     (-1: none), xlim[s] its limit */
  int n_xdas;
  int* xsub;
  int xlim[128];
} oracle_t;

static int64_t binom_tab[72][72];

static void init_binom(void) {
  static int done = 0;
  if (done) return;
  for (int n = 0; n < 72; ++n)
    for (int k = 0; k < 72; ++k)
      binom_tab[n][k] = (k == 0) ? 1 : (n == 0 ? 0 : binom_tab[n - 1][k - 1] + binom_tab[n - 1][k]);
  done = 1;
}

static int64_t binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (n < 72) return binom_tab[n][k];
  int64_t r = 1;   /* larger n only occurs with k <= 2 (core / virtual tuples) */
  for (int j = 1; j <= k; ++j) r = r * (n - k + j) / j;
  return r;
}

/* Neumaier compensated sum in long double */
typedef struct {
  long double s, c;
} ksum_t;

static void kadd(ksum_t* k, long double x) {
  long double t = k->s + x;
  if (fabsl(k->s) >= fabsl(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}

static long double kval(const ksum_t* k) { return k->s + k->c; }

/* ---------------- integrals ---------------- */

static cplx eri_direct(const oracle_t* P, int p, int q, int r, int s) {
  const size_t nn = (size_t)P->n * P->n;
  cplx acc = 0;
  for (int l = 0; l < P->L; ++l)
    acc += P->w[l] * P->B[l * nn + (size_t)p * P->n + q] * P->B[l * nn + (size_t)r * P->n + s];
  return acc;
}

/* chemists' (pq|rs) */
static cplx eri(const oracle_t* P, int p, int q, int r, int s) {
  if (P->eri) {
    size_t n = P->n;
    return P->eri[((p * n + q) * n + r) * n + s];
  }
  return eri_direct(P, p, q, r, s);
}

/* <pq||rs> = <pq|rs> - <pq|sr> = (pr|qs) - (ps|qr) */
static cplx asym(const oracle_t* P, int p, int q, int r, int s) {
  return eri(P, p, r, q, s) - eri(P, p, s, q, r);
}

/* ---------------- bitsets ---------------- */

static inline int det_get(const det_t* d, int p) { return (d->w[p >> 6] >> (p & 63)) & 1; }
static inline void det_set(det_t* d, int p) { d->w[p >> 6] |= (1ull << (p & 63)); }
static inline void det_clr(det_t* d, int p) { d->w[p >> 6] &= ~(1ull << (p & 63)); }

static int det_below(const det_t* d, int p) {
  int c = 0;
  for (int k = 0; k < (p >> 6); ++k) c += __builtin_popcountll(d->w[k]);
  uint64_t m = (p & 63) ? (d->w[p >> 6] & ((1ull << (p & 63)) - 1)) : 0;
  return c + __builtin_popcountll(m);
}

/* a_q |d>: returns 0 when q is empty, else flips the sign for the spinors below q. */
static int apply_ann(det_t* d, int q, int* sign) {
  if (!det_get(d, q)) return 0;
  if (det_below(d, q) & 1) *sign = -*sign;
  det_clr(d, q);
  return 1;
}

static int apply_cre(det_t* d, int p, int* sign) {
  if (det_get(d, p)) return 0;
  if (det_below(d, p) & 1) *sign = -*sign;
  det_set(d, p);
  return 1;
}

/* ---------------- Slater-Condon ---------------- */

static double hdiag(const oracle_t* P, const det_t* K) {
  int occ[1280], no = 0;
  for (int p = 0; p < P->n; ++p)
    if (det_get(K, p)) occ[no++] = p;
  double e = 0;
  for (int i = 0; i < no; ++i) e += creal(P->h[(size_t)occ[i] * P->n + occ[i]]);
  for (int i = 0; i < no; ++i)
    for (int j = 0; j < no; ++j) e += 0.5 * P->G[(size_t)occ[i] * P->n + occ[j]];
  return e;
}

/* <K|H|L> for determinants with the same electron count. */
static cplx hmat(const oracle_t* P, const det_t* K, const det_t* L) {
  int pk[3], ql[3], np = 0, nq = 0;
  for (int k = 0; k < MAXW; ++k) {
    uint64_t a = K->w[k] & ~L->w[k], b = L->w[k] & ~K->w[k];
    while (a) {
      int bit = __builtin_ctzll(a);
      a &= a - 1;
      if (np < 3) pk[np] = 64 * k + bit;
      ++np;
    }
    while (b) {
      int bit = __builtin_ctzll(b);
      b &= b - 1;
      if (nq < 3) ql[nq] = 64 * k + bit;
      ++nq;
    }
  }
  if (np != nq || np > 2) return 0;
  if (np == 0) return hdiag(P, K);
  if (np == 1) {
    int p = pk[0], q = ql[0], sign = 1;
    det_t t = *L;
    apply_ann(&t, q, &sign);
    apply_cre(&t, p, &sign);
    cplx v = P->h[(size_t)p * P->n + q];
    for (int r = 0; r < P->n; ++r)
      if (det_get(&t, r) && r != p) v += asym(P, p, r, q, r);
    return sign * v;
  }
  /* two differences: <K| a+_p1 a+_p2 a_q2 a_q1 |L> <p1 p2||q1 q2> */
  int sign = 1;
  det_t t = *L;
  apply_ann(&t, ql[0], &sign);
  apply_ann(&t, ql[1], &sign);
  apply_cre(&t, pk[1], &sign);
  apply_cre(&t, pk[0], &sign);
  return sign * asym(P, pk[0], pk[1], ql[0], ql[1]);
}

/* ---------------- P-space addressing ---------------- */

static int pattern_index(const oracle_t* P, const int* occ) {
  for (int k = 0; k < P->n_pat; ++k) {
    int same = 1;
    for (int s = 0; s < P->n_das; ++s) same &= (P->pat[k][s] == occ[s]);
    if (same) return k;
  }
  return -1;
}

/* address of an active string (active-local bits) in P, or -1 */
static int64_t p_address_active(const oracle_t* P, uint64_t a) {
  int occ[MAXDAS];
  for (int s = 0; s < P->n_das; ++s) {
    uint64_t m = (P->das_size[s] == 64) ? ~0ull : (((1ull << P->das_size[s]) - 1) << P->das_off[s]);
    occ[s] = __builtin_popcountll(a & m);
  }
  int k = pattern_index(P, occ);
  if (k < 0) return -1;
  int64_t addr = P->pat_off[k], stride = 1;
  for (int s = 0; s < P->n_das; ++s) {
    int64_t rank = 0;
    int j = 0;
    for (int t = 0; t < P->das_size[s]; ++t)
      if ((a >> (P->das_off[s] + t)) & 1) rank += binom(t, ++j);
    addr += rank * stride;
    stride *= binom(P->das_size[s], occ[s]);
  }
  return addr;
}

static void make_det(const oracle_t* P, det_t* d, const int* holes, int nh, uint64_t act,
                     const int* parts, int np) {
  memset(d, 0, sizeof(*d));
  for (int k = 0; k < P->n_core; ++k) det_set(d, k);
  for (int i = 0; i < nh; ++i) det_clr(d, holes[i]);
  for (int t = 0; t < P->n_act; ++t)
    if ((act >> t) & 1) det_set(d, P->a0 + t);
  for (int i = 0; i < np; ++i) det_set(d, parts[i]);
}

static void build_patterns(oracle_t* P) {
  /* lexicographic enumeration, n_1 most significant */
  int cur[MAXDAS];
  P->n_pat = 0;
  int64_t off = 0;
  /* odometer over n_1..n_k */
  for (int s = 0; s < P->n_das; ++s) cur[s] = P->das_min[s];
  for (;;) {
    int sum = 0, ok = 1;
    for (int s = 0; s < P->n_das; ++s) {
      sum += cur[s];
      if (cur[s] > P->das_size[s]) ok = 0;
    }
    if (ok && sum == P->n_elec && P->n_pat < MAXPAT) {
      memcpy(P->pat[P->n_pat], cur, sizeof(int) * P->n_das);
      P->pat_off[P->n_pat] = off;
      int64_t cnt = 1;
      for (int s = 0; s < P->n_das; ++s) cnt *= binom(P->das_size[s], cur[s]);
      off += cnt;
      P->n_pat++;
    }
    int s = P->n_das - 1;
    while (s >= 0) {
      if (cur[s] < P->das_max[s]) {
        cur[s]++;
        break;
      }
      cur[s] = P->das_min[s];
      --s;
    }
    if (s < 0) break;
  }
  P->pat_off[P->n_pat] = off;
}

/* ---------------- API ---------------- */

static void build_pstr(oracle_t* P);


void* oracle_create(const oracle_desc* d) {
  init_binom();
  oracle_t* P = (oracle_t*)calloc(1, sizeof(oracle_t));
  P->n_core = d->n_core;
  P->n_act = d->n_act;
  P->n_virt = d->n_virt;
  P->n = d->n_core + d->n_act + d->n_virt;
  P->n_elec = d->n_elec;
  P->a0 = d->n_core;
  P->v0 = d->n_core + d->n_act;
  P->n_das = d->n_das;
  int off = 0;
  for (int s = 0; s < d->n_das; ++s) {
    P->das_size[s] = d->das_size[s];
    P->das_min[s] = d->das_min[s];
    P->das_max[s] = d->das_max[s];
    P->das_off[s] = off;
    off += d->das_size[s];
  }
  int n = P->n;
  P->frozen = (unsigned char*)malloc(n);
  memcpy(P->frozen, d->frozen, n);
  P->h = (cplx*)malloc(sizeof(cplx) * n * n);
  memcpy(P->h, d->h, sizeof(cplx) * n * n);
  P->L = d->L;
  P->B = (const cplx*)d->B;
  P->w = (double*)malloc(sizeof(double) * (d->L > 0 ? d->L : 1));
  memcpy(P->w, d->w, sizeof(double) * d->L);
  P->b = d->level_shift_b;
  P->n_threads = d->n_threads;
#ifdef _OPENMP
  if (P->n_threads > 0) omp_set_num_threads(P->n_threads);
#endif
  if (d->use_eri_cache) {
    size_t n4 = (size_t)n * n * n * n;
    P->eri = (cplx*)malloc(sizeof(cplx) * n4);
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s)
            P->eri[(((size_t)p * n + q) * n + r) * n + s] = eri_direct(P, p, q, r, s);
  }
  P->G = (double*)malloc(sizeof(double) * n * n);
#pragma omp parallel for schedule(dynamic)
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) P->G[(size_t)p * n + q] = creal(asym(P, p, q, p, q));
  build_patterns(P);
  build_pstr(P);
  P->corr_core = (int*)malloc(sizeof(int) * (P->n_core + 1));
  P->corr_virt = (int*)malloc(sizeof(int) * (P->n_virt + 1));
  for (int k = 0; k < P->n_core; ++k)
    if (!P->frozen[k]) P->corr_core[P->ncc++] = k;
  for (int v = P->v0; v < n; ++v)
    if (!P->frozen[v]) P->corr_virt[P->nvc++] = v;
  P->xsub = (int*)malloc(sizeof(int) * n);
  for (int p = 0; p < n; ++p) P->xsub[p] = -1;
  P->n_xdas = 0;
  return P;
}

void oracle_destroy(void* vp) {
  oracle_t* P = (oracle_t*)vp;
  if (!P) return;
  free(P->frozen);
  free(P->xsub);
  free(P->h);
  free(P->w);
  free(P->eri);
  free(P->G);
  free(P->c);
  free(P->corr_core);
  free(P->corr_virt);
  free(P->pstr);
  free(P);
}

int64_t oracle_np(void* vp) { return ((oracle_t*)vp)->pat_off[((oracle_t*)vp)->n_pat]; }

void oracle_set_c(void* vp, const double* c, int n_roots) {
  oracle_t* P = (oracle_t*)vp;
  int64_t np = oracle_np(P);
  free(P->c);
  P->n_roots = n_roots;
  P->c = (cplx*)malloc(sizeof(cplx) * n_roots * np);
  memcpy(P->c, c, sizeof(cplx) * n_roots * np);
}

/* Gosper's hack: next bit pattern with the same popcount */
static uint64_t next_comb(uint64_t x) {
  uint64_t c = x & (~x + 1), r = x + c;
  return (((r ^ x) >> 2) / c) | r;
}

/* every active string with ne electrons, in increasing integer order */
#define FOR_STRINGS(var, nbits, ne)                                                 \
  for (uint64_t var = ((ne) == 0 ? 0 : ((1ull << (ne)) - 1)), _lim = 1ull << (nbits); \
       (ne) == 0 ? (var == 0) : (var < _lim); var = (ne) == 0 ? 1 : next_comb(var))

static void build_pstr(oracle_t* P) {
  int64_t np = P->pat_off[P->n_pat];
  P->pstr = (uint64_t*)calloc((size_t)(np > 0 ? np : 1), sizeof(uint64_t));
  FOR_STRINGS(A, P->n_act, P->n_elec) {
    int64_t a = p_address_active(P, A);
    if (a >= 0) P->pstr[a] = A;
  }
}

/* Core / virtual DAS subspaces with hole / particle limits (Sec. 2.4, Fig. 1;
   the excitation restrictions of the categories): core subspace s (a block
   of consecutive core spinors) admits at most cmax[s] holes, virtual
   subspace s at most vmax[s] particles.  n_c = n_v = 0 removes them. */
void oracle_set_external_das(void* vp, int n_c, const int* csize, const int* cmax, int n_v, const int* vsize,
                             const int* vmax) {
  oracle_t* P = (oracle_t*)vp;
  for (int p = 0; p < P->n; ++p) P->xsub[p] = -1;
  int at = 0, s = 0;
  for (int k = 0; k < n_c; ++k, ++s) {
    for (int q = 0; q < csize[k]; ++q) P->xsub[at++] = s;
    P->xlim[s] = cmax[k];
  }
  at = P->v0;
  for (int k = 0; k < n_v; ++k, ++s) {
    for (int q = 0; q < vsize[k]; ++q) P->xsub[at++] = s;
    P->xlim[s] = vmax[k];
  }
  P->n_xdas = s;
}

/* Does the external determinant (holes, particles) respect the subspace
   limits?  Counts the holes / particles that fall in each subspace. */
static int external_allowed(const oracle_t* P, const int* holes, int nh, const int* parts, int np) {
  if (P->n_xdas == 0) return 1;
  int cnt[128] = {0};
  for (int k = 0; k < nh; ++k)
    if (P->xsub[holes[k]] >= 0) cnt[P->xsub[holes[k]]]++;
  for (int k = 0; k < np; ++k)
    if (P->xsub[parts[k]] >= 0) cnt[P->xsub[parts[k]]]++;
  for (int s = 0; s < P->n_xdas; ++s)
    if (cnt[s] > P->xlim[s]) return 0;
  return 1;
}

/* P determinants connected to determinant K, for each L: <K|H|L>. */
typedef void (*visit_fn)(void* ctx, int64_t addr, cplx hkl);

static void subset_of(const int* list, int nlist, int k, int64_t idx, int* out) {
  /* idx-th k-subset (k <= 2) of list in lexicographic order */
  if (k == 0) return;
  if (k == 1) {
    out[0] = list[idx];
    return;
  }
  for (int a = 0; a < nlist; ++a) {
    int64_t cnt = nlist - a - 1;
    if (idx < cnt) {
      out[0] = list[a];
      out[1] = list[a + 1 + idx];
      return;
    }
    idx -= cnt;
  }
}

/* All P determinants within two substitutions of K: K has nh core holes and
 * active string A (the virtual particles of K are never occupied in P).
 * A P determinant L has the core full and active string A' = (A - R) + X with
 * X outside A and R inside A; |L - K| = nh + |X| <= 2 and |A'| = n_elec fix
 * |R| = |A| + |X| - n_elec. */
static void for_connected(const oracle_t* P, const det_t* K, int nh, uint64_t A, visit_fn f, void* ctx) {
  int na = __builtin_popcountll(A);
  int cl[64], al[64], ncl = 0, nal = 0;
  for (int t = 0; t < P->n_act; ++t) {
    if ((A >> t) & 1) al[nal++] = t;
    else cl[ncl++] = t;
  }
  for (int nx = 0; nx + nh <= 2; ++nx) {
    int nr = na + nx - P->n_elec;
    if (nr < 0 || nr > na || nr > 2) continue;
    int64_t xcount = binom(ncl, nx), rcount = binom(nal, nr);
    for (int64_t xs = 0; xs < xcount; ++xs) {
      int xi[2];
      subset_of(cl, ncl, nx, xs, xi);
      uint64_t X = 0;
      for (int k = 0; k < nx; ++k) X |= 1ull << xi[k];
      for (int64_t rs = 0; rs < rcount; ++rs) {
        int ri[2];
        subset_of(al, nal, nr, rs, ri);
        uint64_t R = 0;
        for (int k = 0; k < nr; ++k) R |= 1ull << ri[k];
        uint64_t Ap = (A & ~R) | X;
        int64_t addr = p_address_active(P, Ap);
        if (addr < 0) continue;
        det_t Ld;
        make_det(P, &Ld, NULL, 0, Ap, NULL, 0);
        f(ctx, addr, hmat(P, K, &Ld));
      }
    }
  }
}

typedef struct {
  const oracle_t* P;
  cplx* V;
  int hit;
} vctx;

static void acc_v(void* vc, int64_t addr, cplx hkl) {
  vctx* x = (vctx*)vc;
  int64_t np = oracle_np((void*)x->P);
  for (int m = 0; m < x->P->n_roots; ++m) x->V[m] += hkl * x->P->c[m * np + addr];
  x->hit = 1;
}

/* E0_m = <Psi_m|H|Psi_m>/<Psi_m|Psi_m> from explicit P H P rows
   (Sec. 2.3: the reference energy of state m). */
int oracle_e0(void* vp, double* E0) {
  oracle_t* P = (oracle_t*)vp;
  int64_t np = oracle_np(P);
  int R = P->n_roots;
  long double* part = (long double*)calloc((size_t)np * R, sizeof(long double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < np; ++a) {
    uint64_t A = P->pstr[a];
    det_t Ld;
    make_det(P, &Ld, NULL, 0, A, NULL, 0);
    cplx V[64] = {0};
    vctx x = {P, V, 0};
    for_connected(P, &Ld, 0, A, acc_v, &x);   /* (H Psi)_L */
    for (int m = 0; m < R; ++m) part[a * R + m] = creal(conj(P->c[m * np + a]) * V[m]);
  }
  for (int m = 0; m < R; ++m) {
    ksum_t num = {0, 0}, den = {0, 0};
    for (int64_t a = 0; a < np; ++a) {
      cplx cl = P->c[m * np + a];
      kadd(&num, part[a * R + m]);
      kadd(&den, (long double)(creal(cl) * creal(cl) + cimag(cl) * cimag(cl)));
    }
    E0[m] = (double)(kval(&num) / kval(&den));
  }
  free(part);
  return 0;
}

typedef struct {
  int64_t row, n;
  int64_t* rows;
  int64_t* cols;
  double* vals;
  int64_t cap, base;
} cooctx;

static void acc_coo(void* vc, int64_t addr, cplx hkl) {
  cooctx* x = (cooctx*)vc;
  int64_t k = x->base + x->n;
  if (x->rows && k < x->cap) {
    x->rows[k] = x->row;
    x->cols[k] = addr;
    x->vals[2 * k] = creal(hkl);
    x->vals[2 * k + 1] = cimag(hkl);
  }
  x->n++;
}

/* Sparse P H P in coordinate form (row = address of L, col = address of L').
   Pass rows == NULL to count the entries. */
int64_t oracle_hpp_coo(void* vp, int64_t* rows, int64_t* cols, double* vals, int64_t cap) {
  oracle_t* P = (oracle_t*)vp;
  int64_t np = oracle_np(P);
  int64_t* cnt = (int64_t*)calloc((size_t)np + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < np; ++a) {
    det_t Ld;
    make_det(P, &Ld, NULL, 0, P->pstr[a], NULL, 0);
    cooctx x = {a, 0, NULL, NULL, NULL, 0, 0};
    for_connected(P, &Ld, 0, P->pstr[a], acc_coo, &x);
    cnt[a + 1] = x.n;
  }
  for (int64_t a = 0; a < np; ++a) cnt[a + 1] += cnt[a];
  int64_t nnz = cnt[np];
  if (rows && nnz <= cap) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < np; ++a) {
      det_t Ld;
      make_det(P, &Ld, NULL, 0, P->pstr[a], NULL, 0);
      cooctx x = {a, 0, rows, cols, vals, cap, cnt[a]};
      for_connected(P, &Ld, 0, P->pstr[a], acc_coo, &x);
    }
  }
  free(cnt);
  return nnz;
}

/* EN term, plain or with the real part of the imaginary level shift */
static double en_term(double v2, double D, double b) {
  if (b == 0.0) return v2 / D;
  double D2 = D * D;
  return v2 * D * D2 / (D2 * D2 + b * b);
}

/* <c_m|c_m>: Sec. 2.3 takes the reference states normalised, so E2 of an
   unnormalised c is E2 of c/|c| (each term divided by <c|c>). */
static double c_norm(const oracle_t* P, int m) {
  int64_t np = oracle_np((void*)P);
  ksum_t s = {0, 0};
  for (int64_t a = 0; a < np; ++a) {
    cplx v = P->c[m * np + a];
    kadd(&s, (long double)(creal(v) * creal(v) + cimag(v) * cimag(v)));
  }
  return (double)kval(&s);
}

/* E2 per root and class (class id 3*h + p), for Psi = c/|c|.  n_coupl[cls]
   counts the external determinants with at least one connected P determinant. */
int oracle_e2(void* vp, const double* E0, double* e2_class, int64_t* n_coupl) {
  oracle_t* P = (oracle_t*)vp;
  int R = P->n_roots;
  for (int i = 0; i < R * NCLASS; ++i) e2_class[i] = 0;
  for (int i = 0; i < NCLASS; ++i) n_coupl[i] = 0;
  for (int h = 0; h <= 2; ++h)
    for (int p = 0; p <= 2; ++p) {
      int ne = P->n_elec + h - p, cls = 3 * h + p;
      if (ne < 0 || ne > P->n_act) continue;
      int64_t nI = binom(P->ncc, h), nS = binom(P->nvc, p), nitem = nI * nS;
      if (nitem == 0) continue;
      ksum_t* part = (ksum_t*)calloc((size_t)nitem * R, sizeof(ksum_t));
      double norm[64];
      for (int m = 0; m < R; ++m) norm[m] = c_norm(P, m);
      int64_t* cnt = (int64_t*)calloc((size_t)nitem, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
      for (int64_t item = 0; item < nitem; ++item) {
        int holes[2], parts[2];
        subset_of(P->corr_core, P->ncc, h, item / nS, holes);
        subset_of(P->corr_virt, P->nvc, p, item % nS, parts);
        if (!external_allowed(P, holes, h, parts, p)) continue; /* outside Q: subspace limits */
        FOR_STRINGS(A, P->n_act, ne) {
          det_t K;
          make_det(P, &K, holes, h, A, parts, p);
          if (h == 0 && p == 0 && p_address_active(P, A) >= 0) continue; /* K in P */
          cplx V[64] = {0};
          vctx x = {P, V, 0};
          for_connected(P, &K, h, A, acc_v, &x);
          if (!x.hit) continue; /* not connected: outside Q */
          cnt[item]++;
          double hkk = hdiag(P, &K);
          for (int m = 0; m < R; ++m) {
            double v2 = creal(V[m]) * creal(V[m]) + cimag(V[m]) * cimag(V[m]);
            kadd(&part[item * R + m], en_term(v2, E0[m] - hkk, P->b) / norm[m]);
          }
        }
      }
      for (int m = 0; m < R; ++m) {
        ksum_t tot = {0, 0};
        for (int64_t item = 0; item < nitem; ++item) kadd(&tot, kval(&part[item * R + m]));
        e2_class[m * NCLASS + cls] = (double)kval(&tot);
      }
      for (int64_t item = 0; item < nitem; ++item) n_coupl[cls] += cnt[item];
      free(part);
      free(cnt);
    }
  return 0;
}

/* V_K and D_K = E0 - H_KK for listed external determinants.
   holes/parts: [nK][2] global spinor indices (unused slots ignored),
   nh/np: [nK] counts, act: [nK] active-local bit strings.
   V: [nK][n_roots] complex interleaved, D: [nK][n_roots]. */
int oracle_couplings(void* vp, const double* E0, int64_t nK, const int* nh, const int* holes,
                     const int* np_, const int* parts, const uint64_t* act, double* V, double* D) {
  oracle_t* P = (oracle_t*)vp;
  int R = P->n_roots;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nK; ++k) {
    det_t K;
    make_det(P, &K, holes + 2 * k, nh[k], act[k], parts + 2 * k, np_[k]);
    cplx Vk[64] = {0};
    vctx x = {P, Vk, 0};
    for_connected(P, &K, nh[k], act[k], acc_v, &x);
    double hkk = hdiag(P, &K);
    for (int m = 0; m < R; ++m) {
      V[2 * (k * R + m)] = creal(Vk[m]);
      V[2 * (k * R + m) + 1] = cimag(Vk[m]);
      D[k * R + m] = E0[m] - hkk;
    }
  }
  return 0;
}

/* Coupling tensors D^x_A = <A|x|Psi_root> (the <K|E_pq|L> C_L factors of
   Sec. 2.4, Eq. sumsigma, restricted to the active space) for listed active
   strings A, by generic operator algebra on full bitsets: the determinant
   |A> (core full, active bits A, virtuals empty) is acted on by x^dagger
   with the creation / annihilation rules above, and <A|x|L> = conj(<L|x^dagger|A>)
   = the sign that action produced when it reaches a P determinant L (0
   otherwise).  Families (rows r):
     0  x = a_t              r = t
     1  x = a+_t             r = t
     2  x = a_u a_t, t < u   r = u (u - 1) / 2 + t
     3  x = a+_t a+_u, t < u r = u (u - 1) / 2 + t
     4  r = 0: x = 1; r = 1 + t n_act + u: x = a+_t a_u
   out: [rows][nA] complex interleaved. */
int oracle_dtable(void* vp, int family, int root, int64_t nA, const uint64_t* A, double* out) {
  oracle_t* P = (oracle_t*)vp;
  const int na = P->n_act;
  const int rows = family <= 1 ? na : family <= 3 ? na * (na - 1) / 2 : 1 + na * na;
  const int64_t np = P->pat_off[P->n_pat];
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < nA; ++g) {
    for (int r = 0; r < rows; ++r) {
      /* x^dagger as a list of (creator?, spinor) applied right to left: ops[0] first */
      int nops = 0, cre[2] = {0, 0}, sp[2] = {0, 0};
      if (family == 0) { cre[0] = 1; sp[0] = r; nops = 1; }
      else if (family == 1) { cre[0] = 0; sp[0] = r; nops = 1; }
      else if (family <= 3) {
        int u = 1;
        while (u * (u + 1) / 2 <= r) ++u;
        const int t = r - u * (u - 1) / 2;
        if (family == 2) { cre[0] = 1; sp[0] = u; cre[1] = 1; sp[1] = t; }  /* (a_u a_t)^+ = a+_t a+_u */
        else { cre[0] = 0; sp[0] = t; cre[1] = 0; sp[1] = u; }           /* (a+_t a+_u)^+ = a_u a_t */
        nops = 2;
      } else if (r > 0) {
        const int t = (r - 1) / na, u = (r - 1) % na;                   /* (a+_t a_u)^+ = a+_u a_t */
        cre[0] = 0; sp[0] = t; cre[1] = 1; sp[1] = u;
        nops = 2;
      }
      det_t d;
      make_det(P, &d, NULL, 0, A[g], NULL, 0);
      int sign = 1, ok = 1;
      for (int k = 0; k < nops && ok; ++k)
        ok = cre[k] ? apply_cre(&d, P->a0 + sp[k], &sign) : apply_ann(&d, P->a0 + sp[k], &sign);
      cplx v = 0;
      if (ok) {
        uint64_t L = 0;
        for (int t = 0; t < na; ++t)
          if (det_get(&d, P->a0 + t)) L |= 1ull << t;
        const int64_t addr = p_address_active(P, L);
        if (addr >= 0 && root < P->n_roots) v = sign * P->c[(size_t)root * np + addr];
      }
      out[2 * ((size_t)r * nA + g)] = creal(v);
      out[2 * ((size_t)r * nA + g) + 1] = cimag(v);
    }
  }
  return 0;
}

/* Size of Q per class by occupation-pattern counting (no determinants are
   built): class (h,p) with active strings of n_elec+h-p electrons whose
   pattern is at most two substitutions from an allowed pattern:
   h + min_{allowed L} sum_s max(0, nL_s - nA_s) <= 2, and (0,0) excludes P. */
int oracle_count_q(void* vp, double* counts) {
  oracle_t* P = (oracle_t*)vp;
  for (int h = 0; h <= 2; ++h)
    for (int p = 0; p <= 2; ++p) {
      int cls = 3 * h + p, ne = P->n_elec + h - p;
      counts[cls] = 0;
      if (ne < 0 || ne > P->n_act) continue;
      /* enumerate patterns of ne electrons */
      int cur[MAXDAS];
      for (int s = 0; s < P->n_das; ++s) cur[s] = 0;
      double tot = 0;
      for (;;) {
        int sum = 0, ok = 1;
        for (int s = 0; s < P->n_das; ++s) {
          sum += cur[s];
          if (cur[s] > P->das_size[s]) ok = 0;
        }
        if (ok && sum == ne) {
          int best = 1 << 30;
          for (int k = 0; k < P->n_pat; ++k) {
            int d = 0;
            for (int s = 0; s < P->n_das; ++s) d += (P->pat[k][s] > cur[s]) ? P->pat[k][s] - cur[s] : 0;
            if (d < best) best = d;
          }
          int inP = (pattern_index(P, cur) >= 0);
          if (h + best <= 2 && !(h == 0 && p == 0 && inP)) {
            double c = 1;
            for (int s = 0; s < P->n_das; ++s) c *= (double)binom(P->das_size[s], cur[s]);
            tot += c;
          }
        }
        int s = P->n_das - 1;
        while (s >= 0) {
          if (cur[s] < P->das_size[s]) {
            cur[s]++;
            break;
          }
          cur[s] = 0;
          --s;
        }
        if (s < 0) break;
      }
      /* (hole, particle) tuples that respect the subspace limits */
      double items = 0;
      const int64_t nI = binom(P->ncc, h), nS = binom(P->nvc, p);
      for (int64_t it = 0; it < nI * nS; ++it) {
        int holes[2], parts[2];
        subset_of(P->corr_core, P->ncc, h, it / nS, holes);
        subset_of(P->corr_virt, P->nvc, p, it % nS, parts);
        items += external_allowed(P, holes, h, parts, p);
      }
      counts[cls] = tot * items;
    }
  return 0;
}

/* Generic matrix element between two full determinants given as bitsets of
   MAXW words (for brute-force checks). */
void oracle_hmat(void* vp, const uint64_t* K, const uint64_t* L, double* out) {
  det_t a, b;
  memcpy(a.w, K, sizeof(a.w));
  memcpy(b.w, L, sizeof(b.w));
  cplx v = hmat((oracle_t*)vp, &a, &b);
  out[0] = creal(v);
  out[1] = cimag(v);
}

int oracle_maxw(void) { return MAXW; }

/* chemists' (pq|rs) as the oracle evaluates it (for the symmetry pins) */
void oracle_eri(void* vp, int p, int q, int r, int s, double* out) {
  cplx v = eri((oracle_t*)vp, p, q, r, s);
  out[0] = creal(v);
  out[1] = cimag(v);
}

/* ---------------- gradient ----------------
 *
 * d(sum_m s_m E2_m) with respect to h, every factor B^L, the factor weights
 * w_L and the reference coefficients c, by explicit accumulation over the
 * same Q H P rows.  With v_K = |V_K|^2/n, D_K = E0 - H_KK, the term
 * f(v, D) = v/D (or v D^3/(D^4+b^2) with the level shift), g_K = df/dv,
 * h_K = df/dD, n = <c|c>:
 *   dE2 = (2/n) Re sum_K g_K conj(V_K) <K|dH|c> + (sum_K h_K / n) <c|dH|c>
 *         - sum_K h_K <K|dH|K>                                   (H part)
 *   cbar = (2/n) H_PQ (g V) - (2/n^2)(sum_K g_K |V_K|^2) c
 *          + (2/n)(sum_K h_K)(H_PP - E0) c                       (c part)
 * Every matrix element <X|H|Y> met with coefficient k adds Re(k d<X|H|Y>):
 * its h entries and chemists' integrals (pq|rs) = sum_L w_L B^L_pq B^L_rs
 * receive k (times the Slater-Condon sign).  For a complex input z the
 * returned gradient is dE/dRe z + i dE/dIm z, projected on Hermitian
 * matrices for h and each B^L (dE = Re sum conj(grad) dz for Hermitian dz).
 */
typedef struct {
  cplx* gh;  /* coefficient of dh_pq: dE = Re sum gh_pq dh_pq */
  cplx* gB;  /* coefficient of dB^L_pq */
  double* gw;
} gacc_t;

static void acc_eri(const oracle_t* P, gacc_t* G, int p, int q, int r, int s, cplx k) {
  const size_t nn = (size_t)P->n * P->n;
  for (int l = 0; l < P->L; ++l) {
    cplx bpq = P->B[l * nn + (size_t)p * P->n + q], brs = P->B[l * nn + (size_t)r * P->n + s];
    G->gB[l * nn + (size_t)p * P->n + q] += k * P->w[l] * brs;
    G->gB[l * nn + (size_t)r * P->n + s] += k * P->w[l] * bpq;
    G->gw[l] += creal(k * bpq * brs);
  }
}

/* <pq||rs> = (pr|qs) - (ps|qr) */
static void acc_asym(const oracle_t* P, gacc_t* G, int p, int q, int r, int s, cplx k) {
  acc_eri(P, G, p, r, q, s, k);
  acc_eri(P, G, p, s, q, r, -k);
}

/* Re(k d<X|H|Y>) into G, following hmat() term by term */
static void acc_elem(const oracle_t* P, gacc_t* G, const det_t* X, const det_t* Y, cplx k) {
  int pk[3], ql[3], np = 0, nq = 0;
  for (int w = 0; w < MAXW; ++w) {
    uint64_t a = X->w[w] & ~Y->w[w], b = Y->w[w] & ~X->w[w];
    while (a) {
      int bit = __builtin_ctzll(a);
      a &= a - 1;
      if (np < 3) pk[np] = 64 * w + bit;
      ++np;
    }
    while (b) {
      int bit = __builtin_ctzll(b);
      b &= b - 1;
      if (nq < 3) ql[nq] = 64 * w + bit;
      ++nq;
    }
  }
  if (np != nq || np > 2) return;
  if (np == 0) {
    int occ[1280], no = 0;
    for (int p = 0; p < P->n; ++p)
      if (det_get(X, p)) occ[no++] = p;
    for (int i = 0; i < no; ++i) G->gh[(size_t)occ[i] * P->n + occ[i]] += k;
    for (int i = 0; i < no; ++i)
      for (int j = i + 1; j < no; ++j) acc_asym(P, G, occ[i], occ[j], occ[i], occ[j], k);
    return;
  }
  if (np == 1) {
    int p = pk[0], q = ql[0], sign = 1;
    det_t t = *Y;
    apply_ann(&t, q, &sign);
    apply_cre(&t, p, &sign);
    cplx ks = k * (double)sign;
    G->gh[(size_t)p * P->n + q] += ks;
    for (int r = 0; r < P->n; ++r)
      if (det_get(&t, r) && r != p) acc_asym(P, G, p, r, q, r, ks);
    return;
  }
  int sign = 1;
  det_t t = *Y;
  apply_ann(&t, ql[0], &sign);
  apply_ann(&t, ql[1], &sign);
  apply_cre(&t, pk[1], &sign);
  apply_cre(&t, pk[0], &sign);
  acc_asym(P, G, pk[0], pk[1], ql[0], ql[1], k * (double)sign);
}

/* df/dv and df/dD of the Epstein-Nesbet term */
static void en_derivs(double v2, double D, double b, double* gv, double* hD) {
  if (b == 0.0) {
    *gv = 1.0 / D;
    *hD = -v2 / (D * D);
    return;
  }
  double D2 = D * D, den = D2 * D2 + b * b;
  *gv = D * D2 / den;
  *hD = v2 * D2 * (3.0 * b * b - D2 * D2) / (den * den);
}

typedef struct {
  const oracle_t* P;
  const det_t* K;
  cplx coefK;      /* (2/n) s g conj(V) summed over roots is root dependent: kept per root below */
  const cplx* kq;  /* [R] (2/n_m) s_m g_K conj(V_K,m) */
  const cplx* kc;  /* [R] (2/n_m) s_m g_K V_K,m  (for cbar) */
  gacc_t* G;
  cplx* gc;        /* [R][np] */
} gctx;

static void grad_visit_q(void* vc, int64_t addr, cplx hkl) {
  gctx* x = (gctx*)vc;
  const oracle_t* P = x->P;
  int64_t np = oracle_np((void*)P);
  cplx k = 0;
  for (int m = 0; m < P->n_roots; ++m) {
    k += x->kq[m] * P->c[m * np + addr];
    x->gc[m * np + addr] += x->kc[m] * conj(hkl);
  }
  det_t Ld;
  make_det(P, &Ld, NULL, 0, P->pstr[addr], NULL, 0);
  acc_elem(P, x->G, x->K, &Ld, k);
}

typedef struct {
  const oracle_t* P;
  const det_t* Lrow;
  int64_t arow;
  const double* kp;  /* [R] s_m sum_h_m / n_m */
  gacc_t* G;
  cplx* hc;          /* [R][np] (H_PP c) accumulation */
} pctx;

static void grad_visit_p(void* vc, int64_t addr, cplx hkl) {
  pctx* x = (pctx*)vc;
  const oracle_t* P = x->P;
  int64_t np = oracle_np((void*)P);
  cplx k = 0;
  for (int m = 0; m < P->n_roots; ++m) {
    k += x->kp[m] * conj(P->c[m * np + x->arow]) * P->c[m * np + addr];
    x->hc[m * np + x->arow] += hkl * P->c[m * np + addr];
  }
  det_t Ld;
  make_det(P, &Ld, NULL, 0, P->pstr[addr], NULL, 0);
  acc_elem(P, x->G, x->Lrow, &Ld, k);
}

/* Gradient of sum_m seed[m] E2_m.  Outputs, complex interleaved unless noted:
   gh [n][n], gB [L][n][n] (factor order of the descriptor), gw [L] (real),
   gc [n_roots][np].  E0 must be the reference energies of c. */
int oracle_grad(void* vp, const double* E0, const double* seed, double* gh_out, double* gB_out, double* gw_out,
                double* gc_out) {
  oracle_t* P = (oracle_t*)vp;
  const int R = P->n_roots, n = P->n;
  const int64_t np = oracle_np(P);
  const size_t nn = (size_t)n * n;
  double norm[64];
  for (int m = 0; m < R; ++m) norm[m] = c_norm(P, m);
  gacc_t G;
  G.gh = (cplx*)calloc(nn, sizeof(cplx));
  G.gB = (cplx*)calloc(nn * (P->L > 0 ? P->L : 1), sizeof(cplx));
  G.gw = (double*)calloc(P->L > 0 ? P->L : 1, sizeof(double));
  cplx* gc = (cplx*)calloc((size_t)R * np, sizeof(cplx));
  cplx* hc = (cplx*)calloc((size_t)R * np, sizeof(cplx));
  double sum_h[64] = {0}, sum_gv[64] = {0};
  /* Q part (serial: the accumulation targets are shared) */
  for (int h = 0; h <= 2; ++h)
    for (int p = 0; p <= 2; ++p) {
      int ne = P->n_elec + h - p;
      if (ne < 0 || ne > P->n_act) continue;
      int64_t nI = binom(P->ncc, h), nS = binom(P->nvc, p);
      for (int64_t item = 0; item < nI * nS; ++item) {
        int holes[2], parts[2];
        subset_of(P->corr_core, P->ncc, h, item / nS, holes);
        subset_of(P->corr_virt, P->nvc, p, item % nS, parts);
        if (!external_allowed(P, holes, h, parts, p)) continue;
        FOR_STRINGS(A, P->n_act, ne) {
          det_t K;
          make_det(P, &K, holes, h, A, parts, p);
          if (h == 0 && p == 0 && p_address_active(P, A) >= 0) continue;
          cplx V[64] = {0};
          vctx x = {P, V, 0};
          for_connected(P, &K, h, A, acc_v, &x);
          if (!x.hit) continue;
          double hkk = hdiag(P, &K);
          cplx kq[64], kc[64];
          double kdiag = 0.0;
          for (int m = 0; m < R; ++m) {
            double v2 = (creal(V[m]) * creal(V[m]) + cimag(V[m]) * cimag(V[m])) / norm[m];
            double gv, hD;
            en_derivs(v2, E0[m] - hkk, P->b, &gv, &hD);
            sum_h[m] += hD;
            sum_gv[m] += gv * v2 * norm[m];
            kq[m] = (2.0 / norm[m]) * seed[m] * gv * conj(V[m]);
            kc[m] = (2.0 / norm[m]) * seed[m] * gv * V[m];
            kdiag += -seed[m] * hD;
          }
          gctx gx = {P, &K, 0, kq, kc, &G, gc};
          for_connected(P, &K, h, A, grad_visit_q, &gx);
          acc_elem(P, &G, &K, &K, kdiag);
        }
      }
    }
  /* P part: (sum_h / n) <c|dH|c>, and (H_PP c) for cbar */
  double kp[64];
  for (int m = 0; m < R; ++m) kp[m] = seed[m] * sum_h[m] / norm[m];
  for (int64_t a = 0; a < np; ++a) {
    det_t Ld;
    make_det(P, &Ld, NULL, 0, P->pstr[a], NULL, 0);
    pctx px = {P, &Ld, a, kp, &G, hc};
    for_connected(P, &Ld, 0, P->pstr[a], grad_visit_p, &px);
  }
  for (int m = 0; m < R; ++m)
    for (int64_t a = 0; a < np; ++a) {
      cplx cv = P->c[m * np + a];
      gc[m * np + a] += -(2.0 / (norm[m] * norm[m])) * seed[m] * sum_gv[m] * cv +
                        (2.0 / norm[m]) * seed[m] * sum_h[m] * (hc[m * np + a] - E0[m] * cv);
    }
  /* gradient = conj(coefficient), Hermitian projection for h and each B^L */
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      cplx v = 0.5 * (conj(G.gh[(size_t)p * n + q]) + G.gh[(size_t)q * n + p]);
      gh_out[2 * ((size_t)p * n + q)] = creal(v);
      gh_out[2 * ((size_t)p * n + q) + 1] = cimag(v);
    }
  for (int l = 0; l < P->L; ++l)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        cplx v = 0.5 * (conj(G.gB[l * nn + (size_t)p * n + q]) + G.gB[l * nn + (size_t)q * n + p]);
        gB_out[2 * (l * nn + (size_t)p * n + q)] = creal(v);
        gB_out[2 * (l * nn + (size_t)p * n + q) + 1] = cimag(v);
      }
  for (int l = 0; l < P->L; ++l) gw_out[l] = G.gw[l];
  memcpy(gc_out, gc, sizeof(cplx) * R * np);
  free(G.gh);
  free(G.gB);
  free(G.gw);
  free(gc);
  free(hc);
  return 0;
}
