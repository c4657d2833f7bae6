/*
 * Plain, slow FP64 CPU oracle for two-phase selected inversion of an SPD
 * block-arrowhead matrix (sTiles, arXiv 2504.19171).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may call this code. It shares nothing with the
 * CUDA library: its own layout, its own loops, no BLAS.
 *
 * Compile with -ffp-contract=off so that every product and sum is rounded
 * separately and results do not depend on the compiler's FMA choices.
 *
 * Matrix model (Sec. III, Fig. 2 case 7): nt band tile columns of size b,
 * lower bandwidth w tiles, and an arrow tile row of height a (index nt).
 * struct(k) = { k+1 .. min(k+w, nt-1) } U { nt  (if a > 0) }.
 * The selected set is the tile pattern of L (case 7), so Sigma is produced
 * on exactly the tiles (i,k), i in {k} U struct(k).
 *
 * Oracle layout (its own, not the library's): tiles are stored row-major,
 * column k (k < nt) holds [ (k,k) b*b | (k+1,k) .. (k+nsub,k) b*b each |
 * (nt,k) a*b ], followed by the corner (nt,nt) a*a.
 *
 * Functions and the passages they follow:
 *   oracle_cholesky   tiled Cholesky A = L L^T on the pattern (Sec. III,
 *                     the factorization the method starts from); POTRF,
 *                     TRSM, SYRK/GEMM per tile column.
 *   oracle_logdet     logdet(A) = 2 sum log L_ii (not in the paper; a
 *                     plain definition).
 *   oracle_selinv     phase 1 (Algorithm 2: L_ii^{-1} and the scaled
 *                     off-diagonal tiles) then phase 2 (Algorithm 3 / the
 *                     recurrences of Sec. III-A and Algorithm 1 restricted
 *                     to the pattern), i from the last tile down to 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Planted-mistake hooks. The tests rebuild this file with -DORACLE_MUTANT=n
 * (n >= 1) to check that the pins catch each mistake; a normal build has
 * ORACLE_MUTANT == 0 and every hook below is inert. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUT(n) (ORACLE_MUTANT == (n))

typedef struct {
  int nt, b, w, a;
  long *colstart; /* nt+1 entries: start of column k; colstart[nt] = corner */
} oshape;

static int nsub(const oshape *s, int k) {
  int m = s->nt - 1 - k;
  return m < s->w ? m : s->w;
}

static int rows_of(const oshape *s, int i) { return i == s->nt ? s->a : s->b; }

static int oshape_init(oshape *s, int nt, int b, int w, int a) {
  s->nt = nt; s->b = b; s->w = w; s->a = a;
  s->colstart = (long *)malloc(sizeof(long) * (size_t)(nt + 1));
  if (!s->colstart) return -1;
  long off = 0;
  for (int k = 0; k < nt; ++k) {
    s->colstart[k] = off;
    off += (long)(1 + nsub(s, k)) * b * b + (long)a * b;
  }
  s->colstart[nt] = off;
  return 0;
}

static void oshape_free(oshape *s) { free(s->colstart); }

/* Total doubles in the oracle layout. */
long oracle_layout_size(int nt, int b, int w, int a) {
  oshape s;
  if (oshape_init(&s, nt, b, w, a)) return -1;
  long n = s.colstart[nt] + (long)a * a;
  oshape_free(&s);
  return n;
}

/* Is tile (i,k), i >= k, in the pattern? */
static int in_pattern(const oshape *s, int i, int k) {
  if (k == s->nt) return i == s->nt && s->a > 0;
  if (i == s->nt) return s->a > 0;
  return i >= k && i - k <= nsub(s, k);
}

/* Offset of tile (i,k) in the oracle layout, or -1 if not in the pattern. */
long oracle_tile_offset(int nt, int b, int w, int a, int i, int k) {
  oshape s;
  if (oshape_init(&s, nt, b, w, a)) return -1;
  long r = -1;
  if (k >= 0 && k <= nt && i >= k && i <= nt && in_pattern(&s, i, k)) {
    if (k == nt) r = s.colstart[nt];
    else if (i == nt) r = s.colstart[k] + (long)(1 + nsub(&s, k)) * b * b;
    else r = s.colstart[k] + (long)(i - k) * b * b;
  }
  oshape_free(&s);
  return r;
}

static double *tile(const oshape *s, double *base, int i, int k) {
  if (k == s->nt) return base + s->colstart[s->nt];
  if (i == s->nt) return base + s->colstart[k] + (long)(1 + nsub(s, k)) * s->b * s->b;
  return base + s->colstart[k] + (long)(i - k) * s->b * s->b;
}

/* struct(k) as an ascending list; returns its length. */
static int struct_of(const oshape *s, int k, int *out) {
  int n = 0;
  if (k == s->nt) return 0;
  for (int i = k + 1; i <= k + nsub(s, k) - (MUT(6) && nsub(s, k) > 0 ? 1 : 0); ++i) out[n++] = i;
  if (s->a > 0) out[n++] = s->nt;
  return n;
}

/* ---- scalar tile kernels, row-major, leading dimension = column count ---- */

/* In-place lower Cholesky of an m x m tile (Cholesky-Banachiewicz order).
 * Returns 0, or the 1-based row of the first non-positive pivot. The strict
 * upper triangle is set to zero. */
static int potrf(double *T, int m) {
  for (int j = 0; j < m; ++j) {
    double d = T[(long)j * m + j];
    for (int k = 0; k < j; ++k) d -= T[(long)j * m + k] * T[(long)j * m + k];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    T[(long)j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double v = T[(long)i * m + j];
      for (int k = 0; k < j; ++k) v -= T[(long)i * m + k] * T[(long)j * m + k];
      T[(long)i * m + j] = v / ljj;
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) T[(long)i * m + j] = 0.0;
  return 0;
}

/* X (r x m) <- X * L^{-T}, L lower m x m: each row x solves L x^T = x^T. */
static void trsm_right_lt(double *X, int r, const double *L, int m) {
  for (int row = 0; row < r; ++row) {
    double *x = X + (long)row * m;
    for (int j = 0; j < m; ++j) {
      double v = x[j];
      for (int k = 0; k < j; ++k) v -= x[k] * (MUT(5) ? L[(long)k * m + j] : L[(long)j * m + k]);
      x[j] = v / L[(long)j * m + j];
    }
  }
}

/* C (r x c) -= A (r x K) * B (c x K)^T */
static void gemm_sub_nt(double *C, int r, int c, const double *A, const double *B, int K) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double acc = 0.0;
      for (int k = 0; k < K; ++k) acc += A[(long)i * K + k] * B[(long)j * K + k];
      C[(long)i * c + j] -= acc;
    }
}

/* Linv = L^{-1} (m x m lower), by forward substitution against I. */
static void trtri_lower(const double *L, double *Linv, int m) {
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < m; ++i) {
      if (i < c) { Linv[(long)i * m + c] = 0.0; continue; }
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[(long)i * m + k] * Linv[(long)k * m + c];
      Linv[(long)i * m + c] = v / L[(long)i * m + i];
    }
  }
}

/* ------------------------------ public API ------------------------------- */

/* Number of tile GEMMs (tile-by-tile products accumulated into a Sigma tile)
 * that the last oracle_selinv call performed in phase 2. */
static long g_phase2_gemms = 0;
long oracle_last_phase2_gemms(void) { return g_phase2_gemms; }

/* Tiled Cholesky in place: on entry T holds A's lower pattern tiles (diagonal
 * tiles full and symmetric), on exit L (strict upper of diagonal tiles zero).
 * Returns 0 or the LAPACK-style 1-based global column of the first failing
 * pivot. */
int oracle_cholesky(int nt, int b, int w, int a, double *T) {
  oshape s;
  if (nt < 1 || b < 1 || w < 0 || a < 0) return -1;
  if (oshape_init(&s, nt, b, w, a)) return -1;
  int *st = (int *)malloc(sizeof(int) * (size_t)(w + 2));
  int info = 0;
  int last = a > 0 ? nt : nt - 1;
  for (int k = 0; k <= last && !info; ++k) {
    int mk = rows_of(&s, k);
    double *Lkk = tile(&s, T, k, k);
    int f = potrf(Lkk, mk); /* POTRF */
    if (f) { info = (int)((long)k * b + f); break; }
    int ns = struct_of(&s, k, st);
    for (int t = 0; t < ns; ++t) /* TRSM */
      trsm_right_lt(tile(&s, T, st[t], k), rows_of(&s, st[t]), Lkk, mk);
    for (int t = 0; t < ns; ++t) /* SYRK / GEMM on the trailing pattern */
      for (int u = 0; u <= t; ++u) {
        int i = st[t], j = st[u];
        gemm_sub_nt(tile(&s, T, i, j), rows_of(&s, i), rows_of(&s, j), tile(&s, T, i, k),
                    tile(&s, T, j, k), mk);
      }
  }
  if (!info) /* the SYRK touched the full diagonal tiles: keep L's upper zero */
    for (int k = 0; k <= last; ++k) {
      int m = rows_of(&s, k);
      double *D = tile(&s, T, k, k);
      for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) D[(long)i * m + j] = 0.0;
    }
  free(st);
  oshape_free(&s);
  return info;
}

/* logdet(A) = 2 * sum over diagonal tiles of log L_dd, summed in order. */
double oracle_logdet(int nt, int b, int w, int a, const double *L) {
  oshape s;
  if (oshape_init(&s, nt, b, w, a)) return NAN;
  double acc = 0.0;
  int last = a > 0 ? nt : nt - 1;
  for (int k = 0; k <= last; ++k) {
    int m = rows_of(&s, k);
    const double *D = tile(&s, (double *)L, k, k);
    for (int d = 0; d < m; ++d) acc += log(D[(long)d * m + d]);
  }
  oshape_free(&s);
  return (MUT(7) ? 1.0 : 2.0) * acc;
}

/* Selected inversion: Sigma on the tile pattern of L.
 * Phase 1 (Algorithm 2): Linv_ii = L_ii^{-1}; U_ki = L_ki Linv_ii, k in
 *   struct(i) (the paper writes U over L in place; the oracle keeps L).
 * Phase 2 (Algorithm 3 with the recurrences of Sec. III-A): for i from the
 *   last tile down to 0,
 *     Sigma_ji = - sum_{k in struct(i)} S_jk U_ki,   j in struct(i),
 *       with S_jk = Sigma_jk (j >= k) or Sigma_kj^T (j < k); as in
 *       Algorithm 1 the k = j term is applied first, then the others in
 *       ascending k;
 *     Sigma_ii = Linv_ii^T Linv_ii - sum_{k in struct(i)} Sigma_ki^T U_ki
 *       (ascending k), then the lower triangle is mirrored to the upper.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_selinv(int nt, int b, int w, int a, const double *Lc, double *S) {
  oshape s;
  if (nt < 1 || b < 1 || w < 0 || a < 0) return -1;
  if (oshape_init(&s, nt, b, w, a)) return -1;
  double *L = (double *)Lc;
  long total = s.colstart[nt] + (long)a * a;
  double *U = (double *)calloc((size_t)total, sizeof(double));
  double *Linv = (double *)calloc((size_t)total, sizeof(double));
  int *st = (int *)malloc(sizeof(int) * (size_t)(w + 2));
  if (!U || !Linv || !st) { free(U); free(Linv); free(st); oshape_free(&s); return -1; }
  memset(S, 0, sizeof(double) * (size_t)total); /* Sigma starts at zero */
  int last = a > 0 ? nt : nt - 1;

  /* Phase 1: independent per tile column. */
  for (int i = 0; i <= last; ++i) {
    int mi = rows_of(&s, i);
    double *Li = tile(&s, Linv, i, i);
    trtri_lower(tile(&s, L, i, i), Li, mi); /* "TRSM(L_ii^T, I)" */
    int ns = struct_of(&s, i, st);
    for (int t = 0; t < ns; ++t) { /* TRMM: U_ki = L_ki Linv_ii */
      int k = st[t], mk = rows_of(&s, k);
      const double *Lki = tile(&s, L, k, i);
      double *Uki = tile(&s, U, k, i);
      for (int r = 0; r < mk; ++r)
        for (int c = 0; c < mi; ++c) {
          double acc = 0.0;
          for (int q = c; q < mi; ++q) acc += Lki[(long)r * mi + q] * Li[(long)q * mi + c];
          Uki[(long)r * mi + c] = acc;
        }
    }
  }

  /* Phase 2: dependent backward sweep. */
  g_phase2_gemms = 0;
  for (int i = last; i >= 0; --i) {
    int mi = rows_of(&s, i);
    int ns = struct_of(&s, i, st);
    /* off-diagonal tiles, j from the last down (the j loop of Algorithm 3) */
    for (int tj = ns - 1; tj >= 0; --tj) {
      int j = st[tj], mj = rows_of(&s, j);
      double *Sji = tile(&s, S, j, i);
      /* k = j term first, then the others ascending */
      for (int pass = 0; pass < 2; ++pass)
        for (int tk = 0; tk < ns; ++tk) {
          int k = st[tk];
          if ((pass == 0) != (k == j)) continue;
          if (MUT(1) && k == s.nt) continue; /* mutant: drop the arrow term */
          int mk = rows_of(&s, k);
          const double *Uki = tile(&s, U, k, i);
          const double *Sx = (j >= k) ? tile(&s, S, j, k) : tile(&s, S, k, j);
          ++g_phase2_gemms;
          for (int r = 0; r < mj; ++r)
            for (int c = 0; c < mi; ++c) {
              double acc = 0.0;
              for (int q = 0; q < mk; ++q) {
                double sjk = (j >= k || MUT(3)) ? Sx[(long)r * mk + q] : Sx[(long)q * mj + r];
                acc += sjk * Uki[(long)q * mi + c];
              }
              Sji[(long)r * mi + c] -= acc;
            }
        }
    }
    /* diagonal tile: LAUUM, then the GEMM updates, then mirror */
    double *Sii = tile(&s, S, i, i);
    const double *Li = tile(&s, Linv, i, i);
    for (int r = 0; r < mi; ++r)
      for (int c = 0; c < mi; ++c) {
        double acc = 0.0;
        int q0 = r > c ? r : c;
        for (int q = q0; q < mi; ++q)
          acc += (MUT(4) ? Li[(long)r * mi + q] : Li[(long)q * mi + r]) * Li[(long)q * mi + c];
        Sii[(long)r * mi + c] = acc;
      }
    for (int tk = 0; tk < ns; ++tk) {
      int k = st[tk], mk = rows_of(&s, k);
      const double *Ski = tile(&s, S, k, i);
      const double *Uki = tile(&s, U, k, i);
      ++g_phase2_gemms;
      for (int r = 0; r < mi; ++r)
        for (int c = 0; c < mi; ++c) {
          double acc = 0.0;
          for (int q = 0; q < mk; ++q) acc += Ski[(long)q * mi + r] * Uki[(long)q * mi + c];
          if (MUT(2)) Sii[(long)r * mi + c] += acc; else /* mutant: sign */
          Sii[(long)r * mi + c] -= acc;
        }
    }
    for (int r = 0; r < mi; ++r)
      for (int c = r + 1; c < mi; ++c) Sii[(long)r * mi + c] = Sii[(long)c * mi + r];
  }
  free(U);
  free(Linv);
  free(st);
  oshape_free(&s);
  return 0;
}
