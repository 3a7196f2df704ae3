/*
 * sph_oracle.c -- plain FP64 CPU oracle of the SPH hot path.
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only callers. The CUDA library shares no
 * code, header, table or helper with this file, and this file includes nothing
 * from it.
 *
 * What it computes (Schaller, Gonnet, Chalk, Draper, PASC '16, Section 2):
 *   - the smoothing kernel W(r,h) (cubic spline, support radius h: Section 2
 *     names h the radius of the sphere of particles considered and leaves the
 *     kernel form open);
 *   - the smoothing length h_i of every particle, chosen so that the weighted
 *     neighbour number N_i(h) = (4 pi / 3) h^3 sum_j W(r_ij, h) equals a fixed
 *     target (Section 2: the number of neighbours is kept roughly constant);
 *   - the density rho_i = sum_{j, r_ij < h_i} m_j W(r_ij, h_i) (Eq. rho),
 *     its derivative d rho_i / d h, and Omega_i = 1 + h_i/(3 rho_i) drho/dh;
 *   - the pressure P_i = rho_i u_i (gamma - 1) and the accelerations and
 *     internal-energy rates of Eqs. (dvdt) and (dudt).
 *
 * Distances are minimum-image distances in the periodic box [0,L_x)x[0,L_y)
 * x[0,L_z). Neighbours are enumerated either by scanning all particles
 * (brute force) or by a periodic k-d tree; both feed the same sums, and the
 * tests check that they find identical neighbour sets.
 *
 * Everything is double precision. OpenMP spreads independent particles over
 * threads; the order of every per-particle sum is the candidate order of the
 * enumeration, nothing is fused or reblocked.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EBOXTOOSMALL (-2)
#define OR_ENONPHYSICAL (-3)
#define OR_ENOMEM (-4)

#define OR_PI 3.14159265358979323846

int or_version(void) { return 1; }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ kernel */

/* Dimensionless cubic spline w(q) and its derivative w'(q), support q < 1:
 *   w(q) = 1 - 6 q^2 + 6 q^3      for 0 <= q < 1/2
 *        = 2 (1 - q)^3            for 1/2 <= q < 1
 *        = 0                      for q >= 1
 * W(r,h) = (8/pi) w(r/h) / h^3 integrates to one over R^3. */
static void w_hat(double q, double *w, double *dw) {
  if (q < 0.5) {
    *w = 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    *dw = -12.0 * q + 18.0 * q * q;
  } else if (q < 1.0) {
    double t = 1.0 - q;
    *w = 2.0 * t * t * t;
    *dw = -6.0 * t * t;
  } else {
    *w = 0.0;
    *dw = 0.0;
  }
}

void or_w_hat(int64_t n, const double *q, double *w, double *dw) {
  for (int64_t k = 0; k < n; ++k) w_hat(q[k], &w[k], &dw[k]);
}

/* W(r,h) = (8/pi) w(r/h) / h^3 */
double or_W(double r, double h) {
  double w, dw;
  w_hat(r / h, &w, &dw);
  return 8.0 / OR_PI * w / (h * h * h);
}

/* dW/dr = (8/pi) w'(r/h) / h^4 */
double or_dWdr(double r, double h) {
  double w, dw;
  w_hat(r / h, &w, &dw);
  return 8.0 / OR_PI * dw / (h * h * h * h);
}

/* dW/dh = -(8/pi) (3 w(q) + q w'(q)) / h^4 */
double or_dWdh(double r, double h) {
  double w, dw, q = r / h;
  w_hat(q, &w, &dw);
  return -8.0 / OR_PI * (3.0 * w + q * dw) / (h * h * h * h);
}

/* ------------------------------------------------------------- geometry */

/* minimum-image displacement d = x_i - x_j in the periodic box */
static void min_image(const double *xi, const double *xj, const double *L, double d[3]) {
  for (int k = 0; k < 3; ++k) {
    double t = xi[k] - xj[k];
    d[k] = t - L[k] * round(t / L[k]);
  }
}

static double norm3(const double d[3]) { return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]); }

/* ------------------------------------------------------- periodic k-d tree */

#define KD_LEAF 16

typedef struct {
  double lo[3], hi[3]; /* bounding box of the node's points */
  double hmax;         /* largest h of the node's points (force queries) */
  int64_t begin, end;  /* index range into perm */
  int64_t left, right; /* children, -1 for a leaf */
} kd_node;

typedef struct {
  const double *x;
  int64_t n;
  double L[3];
  int64_t *perm;
  kd_node *node;
  int64_t n_node, cap;
} kd_tree;

/* Put the k-th smallest coordinate (dimension d) of perm[lo..hi) at index k,
 * smaller-or-equal keys before it, greater-or-equal after (quickselect). */
static void kd_select(int64_t *p, int64_t lo, int64_t hi, int64_t k, const double *x, int d) {
  hi -= 1;
  while (hi > lo) {
    int64_t mid = lo + (hi - lo) / 2;
    double a = x[3 * p[lo] + d], b = x[3 * p[mid] + d], c = x[3 * p[hi] + d];
    double pivot = (a < b) ? ((b < c) ? b : ((a < c) ? c : a)) : ((a < c) ? a : ((b < c) ? c : b));
    int64_t i = lo, j = hi;
    while (i <= j) {
      while (x[3 * p[i] + d] < pivot) ++i;
      while (x[3 * p[j] + d] > pivot) --j;
      if (i <= j) {
        int64_t t = p[i];
        p[i] = p[j];
        p[j] = t;
        ++i;
        --j;
      }
    }
    if (k <= j)
      hi = j;
    else if (k >= i)
      lo = i;
    else
      break;
  }
}

static int64_t kd_alloc(kd_tree *t) {
  int64_t id = __atomic_fetch_add(&t->n_node, 1, __ATOMIC_RELAXED);
  return (id < t->cap) ? id : -1;
}

static void kd_build_node(kd_tree *t, int64_t id, int64_t begin, int64_t end) {
  kd_node *nd = &t->node[id];
  nd->begin = begin;
  nd->end = end;
  nd->left = nd->right = -1;
  nd->hmax = 0.0;
  for (int k = 0; k < 3; ++k) {
    nd->lo[k] = INFINITY;
    nd->hi[k] = -INFINITY;
  }
  for (int64_t s = begin; s < end; ++s) {
    const double *xp = &t->x[3 * t->perm[s]];
    for (int k = 0; k < 3; ++k) {
      if (xp[k] < nd->lo[k]) nd->lo[k] = xp[k];
      if (xp[k] > nd->hi[k]) nd->hi[k] = xp[k];
    }
  }
  if (end - begin <= KD_LEAF) return;
  int d = 0;
  double ext = nd->hi[0] - nd->lo[0];
  for (int k = 1; k < 3; ++k)
    if (nd->hi[k] - nd->lo[k] > ext) {
      ext = nd->hi[k] - nd->lo[k];
      d = k;
    }
  if (ext <= 0.0) return; /* all points coincide: keep as a leaf */
  int64_t mid = begin + (end - begin) / 2;
  kd_select(t->perm, begin, end, mid, t->x, d);
  int64_t l = kd_alloc(t), r = kd_alloc(t);
  if (l < 0 || r < 0) return; /* capacity is sized so this never happens */
  nd->left = l;
  nd->right = r;
  if (end - begin > (1 << 16)) {
#pragma omp task
    kd_build_node(t, l, begin, mid);
#pragma omp task
    kd_build_node(t, r, mid, end);
#pragma omp taskwait
  } else {
    kd_build_node(t, l, begin, mid);
    kd_build_node(t, r, mid, end);
  }
}

static int kd_build(kd_tree *t, const double *x, int64_t n, const double *L) {
  t->x = x;
  t->n = n;
  for (int k = 0; k < 3; ++k) t->L[k] = L[k];
  t->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  t->cap = 4 * (n / KD_LEAF + 1) + 64;
  t->node = (kd_node *)malloc(sizeof(kd_node) * (size_t)t->cap);
  t->n_node = 0;
  if (!t->perm || !t->node) {
    free(t->perm);
    free(t->node);
    return OR_ENOMEM;
  }
  for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
  int64_t root = kd_alloc(t);
#pragma omp parallel
#pragma omp single
  kd_build_node(t, root, 0, n);
  return OR_OK;
}

static void kd_free(kd_tree *t) {
  free(t->perm);
  free(t->node);
}

/* hmax of every node; children always have larger ids than their parent */
static void kd_set_h(kd_tree *t, const double *h) {
  for (int64_t id = t->n_node - 1; id >= 0; --id) {
    kd_node *nd = &t->node[id];
    if (nd->left < 0) {
      double m = 0.0;
      for (int64_t s = nd->begin; s < nd->end; ++s)
        if (h[t->perm[s]] > m) m = h[t->perm[s]];
      nd->hmax = m;
    } else {
      double a = t->node[nd->left].hmax, b = t->node[nd->right].hmax;
      nd->hmax = a > b ? a : b;
    }
  }
}

static double box_dist2(const kd_node *nd, const double q[3]) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    double d = 0.0;
    if (q[k] < nd->lo[k])
      d = nd->lo[k] - q[k];
    else if (q[k] > nd->hi[k])
      d = q[k] - nd->hi[k];
    s += d * d;
  }
  return s;
}

/* ------------------------------------------------------ candidate buffer */

typedef struct {
  int64_t *j;
  double *r;
  double (*d)[3];
  int64_t n, cap;
  int overflow;
} cand_buf;

static int cand_push(cand_buf *b, int64_t j, double r, const double d[3]) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 256;
    int64_t *nj = (int64_t *)realloc(b->j, sizeof(int64_t) * (size_t)nc);
    if (nj) b->j = nj;
    double *nr = (double *)realloc(b->r, sizeof(double) * (size_t)nc);
    if (nr) b->r = nr;
    double(*ndd)[3] = (double(*)[3])realloc(b->d, sizeof(double[3]) * (size_t)nc);
    if (ndd) b->d = ndd;
    if (!nj || !nr || !ndd) return OR_ENOMEM;
    b->cap = nc;
  }
  b->j[b->n] = j;
  b->r[b->n] = r;
  b->d[b->n][0] = d[0];
  b->d[b->n][1] = d[1];
  b->d[b->n][2] = d[2];
  b->n++;
  return OR_OK;
}

static void cand_free(cand_buf *b) {
  free(b->j);
  free(b->r);
  free(b->d);
}

/* Neighbour enumeration. Collects every j (j == i included) whose
 * minimum-image distance to particle i is below R_i -- or, in "force" mode,
 * below max(R_i, h_j). `limit` > 0 aborts the collection (overflow = 1) once
 * more than `limit` candidates are found. The distance test uses min_image()
 * in both modes. */
typedef struct {
  const double *x;
  int64_t n;
  const double *L;
  const kd_tree *tree; /* NULL: brute force */
  const double *h;     /* force mode: per-particle h, else NULL */
} finder;

static int consider(const finder *f, int64_t i, int64_t j, double R, cand_buf *b, int64_t limit) {
  double d[3];
  min_image(&f->x[3 * i], &f->x[3 * j], f->L, d);
  double r = norm3(d);
  double reach = R;
  if (f->h && f->h[j] > reach) reach = f->h[j];
  if (r < reach) {
    if (limit > 0 && b->n >= limit) {
      b->overflow = 1;
      return OR_OK;
    }
    return cand_push(b, j, r, d);
  }
  return OR_OK;
}

static int collect(const finder *f, int64_t i, double R, cand_buf *b, int64_t limit) {
  b->n = 0;
  b->overflow = 0;
  if (!f->tree) {
    for (int64_t j = 0; j < f->n && !b->overflow; ++j) {
      int rc = consider(f, i, j, R, b, limit);
      if (rc) return rc;
    }
    return OR_OK;
  }
  const kd_tree *t = f->tree;
  const double *p = &f->x[3 * i];
  double reach = R;
  if (f->h && t->node[0].hmax > reach) reach = t->node[0].hmax;
  int64_t stack[256];
  for (int sx = -1; sx <= 1; ++sx)
    for (int sy = -1; sy <= 1; ++sy)
      for (int sz = -1; sz <= 1; ++sz) {
        double q[3] = {p[0] + sx * t->L[0], p[1] + sy * t->L[1], p[2] + sz * t->L[2]};
        if (box_dist2(&t->node[0], q) >= reach * reach) continue;
        int top = 0;
        stack[top++] = 0;
        while (top > 0 && !b->overflow) {
          const kd_node *nd = &t->node[stack[--top]];
          double rr = R;
          if (f->h && nd->hmax > rr) rr = nd->hmax;
          if (box_dist2(nd, q) >= rr * rr) continue;
          if (nd->left < 0) {
            for (int64_t s = nd->begin; s < nd->end; ++s) {
              int64_t j = t->perm[s];
              /* a j reached through two images is the same minimum image only
               * once: keep it under the image that realises the minimum */
              double dq[3] = {q[0] - f->x[3 * j], q[1] - f->x[3 * j + 1], q[2] - f->x[3 * j + 2]};
              int same = 1;
              for (int k = 0; k < 3; ++k)
                if (fabs(dq[k]) > 0.5 * t->L[k]) same = 0;
              if (!same) continue;
              int rc = consider(f, i, j, R, b, limit);
              if (rc) return rc;
            }
          } else {
            stack[top++] = nd->left;
            stack[top++] = nd->right;
          }
        }
        if (b->overflow) return OR_OK;
      }
  return OR_OK;
}

/* -------------------------------------------------- neighbour-number sums */

/* Sums over the candidates at smoothing length h (only r < h contributes):
 *   nw   = (32/3) sum_j w(q)                 weighted neighbour number
 *   dnw  = -(32 / (3 h)) sum_j q w'(q)       its h derivative
 *   rho  = (8/pi) h^-3 sum_j m_j w(q)        Eq. (rho)
 *   drho = -(8/pi) h^-4 sum_j m_j (3 w + q w')
 *   cnt  = #{j != i : r < h}                 (self excluded)               */
typedef struct {
  double nw, dnw, rho, drho;
  int64_t cnt;
} dens_sums;

static dens_sums sums_at(const cand_buf *b, int64_t i, double h, const double *m) {
  dens_sums s = {0, 0, 0, 0, 0};
  double sw = 0, sqdw = 0, smw = 0, smdh = 0;
  for (int64_t k = 0; k < b->n; ++k) {
    double r = b->r[k];
    if (!(r < h)) continue;
    double q = r / h, w, dw;
    w_hat(q, &w, &dw);
    double mj = m ? m[b->j[k]] : 1.0;
    sw += w;
    sqdw += q * dw;
    smw += mj * w;
    smdh += mj * (3.0 * w + q * dw);
    if (b->j[k] != i) s.cnt++;
  }
  s.nw = 32.0 / 3.0 * sw;
  s.dnw = -32.0 / (3.0 * h) * sqdw;
  s.rho = 8.0 / OR_PI * smw / (h * h * h);
  s.drho = -8.0 / OR_PI * smdh / (h * h * h * h);
  return s;
}

static double min3(const double *L) {
  double a = L[0] < L[1] ? L[0] : L[1];
  return a < L[2] ? a : L[2];
}

/* Smoothing length of particle i: the unique h with N_i(h) = n_ngb.
 * N_i is continuous and non-decreasing in h (every w(r/h) grows with h),
 * equals 32/3 < n_ngb for h -> 0 (self term only), so the root is bracketed
 * once N_i(R) >= n_ngb for a search radius R. Safeguarded Newton inside the
 * bracket, stopped at |dh| <= tol * h. */
static int solve_h(const finder *f, int64_t i, double h0, double n_ngb, double tol,
                   cand_buf *b, double *h_out, int *iters) {
  const double Rmax = min3(f->L) / 3.0;
  double R = h0 > 0 ? h0 : Rmax * 0.01;
  if (R > Rmax) R = Rmax;
  double lo = 0.0;      /* N(lo) < n_ngb known */
  int64_t limit = 1024; /* candidate cap while R may be far too large */
  for (int guard = 0; guard < 400; ++guard) {
    int rc = collect(f, i, R, b, limit);
    if (rc) return rc;
    if (b->overflow) {
      /* far more candidates than a root radius holds: shrink the search
       * radius (the root is unique, so only the search path changes) */
      if (0.35 * R > lo) {
        R *= 0.35;
      } else {
        limit = 0;
      }
      continue;
    }
    dens_sums s = sums_at(b, i, R, NULL);
    if (s.nw < n_ngb) {
      lo = R;
      if (R >= Rmax) return OR_EBOXTOOSMALL;
      R = 2.0 * R < Rmax ? 2.0 * R : Rmax;
      continue;
    }
    break;
  }
  double hi = R;
  double h = (h0 > lo && h0 < hi) ? h0 : 0.5 * (lo + hi);
  int it = 0;
  for (; it < 300; ++it) {
    dens_sums s = sums_at(b, i, h, NULL);
    double fval = s.nw - n_ngb;
    if (fval == 0.0) break;
    if (fval < 0.0)
      lo = h;
    else
      hi = h;
    double hn = h - fval / s.dnw;
    if (!(s.dnw > 0.0) || !(hn > lo) || !(hn < hi)) hn = 0.5 * (lo + hi);
    double step = fabs(hn - h);
    h = hn;
    if (step <= tol * h || (hi - lo) <= tol * h) break;
  }
  *h_out = h;
  *iters = it + 1;
  return OR_OK;
}

/* ------------------------------------------------------------ public API */

static int check_box(const double *L) {
  for (int k = 0; k < 3; ++k)
    if (!(L[k] > 0.0)) return OR_EINVAL;
  return OR_OK;
}

/* Neighbour lists for pins: for every i, all j != i with r_ij < R[i].
 * counts[i] receives the count; if `idx` is non-NULL, offs (n+1) must hold the
 * exclusive prefix of counts and idx receives the j's (enumeration order). */
int or_neighbours(int64_t n, const double *x, const double *L, const double *R, int use_tree,
                  int64_t *counts, const int64_t *offs, int64_t *idx) {
  if (n < 0 || check_box(L)) return OR_EINVAL;
  kd_tree t;
  int rc = OR_OK;
  if (use_tree && (rc = kd_build(&t, x, n, L))) return rc;
  finder f = {x, n, L, use_tree ? &t : NULL, NULL};
#pragma omp parallel reduction(min : rc)
  {
    cand_buf b = {0};
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      int r = collect(&f, i, R[i], &b, 0);
      if (r) {
        rc = r;
        continue;
      }
      int64_t c = 0;
      for (int64_t k = 0; k < b.n; ++k)
        if (b.j[k] != i) {
          if (idx) idx[offs[i] + c] = b.j[k];
          ++c;
        }
      counts[i] = c;
    }
    cand_free(&b);
  }
  if (use_tree) kd_free(&t);
  return rc;
}

/* Density sums at fixed smoothing lengths h (no root finding). */
int or_density_fixed_h(int64_t n, const double *x, const double *m, const double *L,
                       const double *h, int use_tree, double *rho, double *drho_dh, double *nw,
                       double *dnw_dh, int64_t *cnt) {
  if (n < 0 || check_box(L)) return OR_EINVAL;
  kd_tree t;
  int rc = OR_OK;
  if (use_tree && (rc = kd_build(&t, x, n, L))) return rc;
  finder f = {x, n, L, use_tree ? &t : NULL, NULL};
#pragma omp parallel reduction(min : rc)
  {
    cand_buf b = {0};
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      int r = collect(&f, i, h[i], &b, 0);
      if (r) {
        rc = r;
        continue;
      }
      dens_sums s = sums_at(&b, i, h[i], m);
      rho[i] = s.rho;
      drho_dh[i] = s.drho;
      nw[i] = s.nw;
      dnw_dh[i] = s.dnw;
      cnt[i] = s.cnt;
    }
    cand_free(&b);
  }
  if (use_tree) kd_free(&t);
  return rc;
}

/* Density stage: solve h_i (N_i(h_i) = n_ngb), then rho_i, drho_i/dh,
 * Omega_i = 1 + h_i / (3 rho_i) drho_i/dh (Section 2). h holds the initial
 * guesses on entry and the roots on exit. If `subset` is non-NULL only those
 * particles are solved (outputs stay indexed by particle id). */
int or_density(int64_t n, const double *x, const double *m, const double *L, double n_ngb,
               double tol, int use_tree, double *h, double *rho, double *drho_dh, double *omega,
               double *nw, int64_t *cnt, int32_t *iters, const int64_t *subset,
               int64_t n_subset) {
  if (n < 0 || check_box(L) || !(n_ngb > 32.0 / 3.0)) return OR_EINVAL;
  kd_tree t;
  int rc = OR_OK;
  if (use_tree && (rc = kd_build(&t, x, n, L))) return rc;
  finder f = {x, n, L, use_tree ? &t : NULL, NULL};
  int64_t count = subset ? n_subset : n;
#pragma omp parallel reduction(min : rc)
  {
    cand_buf b = {0};
#pragma omp for schedule(dynamic, 32)
    for (int64_t s = 0; s < count; ++s) {
      int64_t i = subset ? subset[s] : s;
      double hi;
      int it = 0;
      int r = solve_h(&f, i, h[i], n_ngb, tol, &b, &hi, &it);
      if (r) {
        rc = r;
        continue;
      }
      /* candidates cover r < R >= h: re-collect exactly at the root */
      r = collect(&f, i, hi, &b, 0);
      if (r) {
        rc = r;
        continue;
      }
      dens_sums d = sums_at(&b, i, hi, m);
      h[i] = hi;
      rho[i] = d.rho;
      drho_dh[i] = d.drho;
      omega[i] = 1.0 + hi / (3.0 * d.rho) * d.drho;
      nw[i] = d.nw;
      cnt[i] = d.cnt;
      iters[i] = it;
      if (!(d.rho > 0.0) || !(omega[i] > 0.0)) rc = OR_ENONPHYSICAL;
    }
    cand_free(&b);
  }
  if (use_tree) kd_free(&t);
  return rc;
}

/* Force stage, Eqs. (dvdt) and (dudt):
 *   A_i   = P_i / (Omega_i rho_i^2),  P_i = rho_i u_i (gamma - 1)
 *   a_i   = - sum_j m_j [A_i dW/dr(r_ij,h_i) + A_j dW/dr(r_ij,h_j)] (x_i - x_j)/r_ij
 *   du_i  =   A_i sum_j m_j dW/dr(r_ij,h_i) (v_i - v_j).(x_i - x_j)/r_ij
 * over j != i with r_ij < max(h_i, h_j) (each term vanishes outside its own
 * support). Coincident pairs (r = 0) contribute nothing: dW/dr -> 0 there.
 * cnt[i] = #{j != i : r_ij < max(h_i, h_j)}. */
int or_force(int64_t n, const double *x, const double *v, const double *m, const double *u,
             const double *h, const double *rho, const double *omega, const double *L,
             double gamma, int use_tree, double *a, double *dudt, int64_t *cnt,
             const int64_t *subset, int64_t n_subset) {
  if (n < 0 || check_box(L)) return OR_EINVAL;
  double *A = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!A) return OR_ENOMEM;
  double hmax = 0.0;
  int rc = OR_OK;
  for (int64_t i = 0; i < n; ++i) {
    double P = rho[i] * u[i] * (gamma - 1.0);
    A[i] = P / (omega[i] * rho[i] * rho[i]);
    if (h[i] > hmax) hmax = h[i];
    if (!(rho[i] > 0.0) || !(omega[i] > 0.0) || !(h[i] > 0.0)) rc = OR_ENONPHYSICAL;
  }
  if (rc) {
    free(A);
    return rc;
  }
  if (hmax >= min3(L) / 3.0) {
    free(A);
    return OR_EBOXTOOSMALL;
  }
  kd_tree t;
  if (use_tree) {
    if ((rc = kd_build(&t, x, n, L))) {
      free(A);
      return rc;
    }
    kd_set_h(&t, h);
  }
  finder f = {x, n, L, use_tree ? &t : NULL, h};
  int64_t count = subset ? n_subset : n;
#pragma omp parallel reduction(min : rc)
  {
    cand_buf b = {0};
#pragma omp for schedule(dynamic, 32)
    for (int64_t s = 0; s < count; ++s) {
      int64_t i = subset ? subset[s] : s;
      int r = collect(&f, i, h[i], &b, 0);
      if (r) {
        rc = r;
        continue;
      }
      double ax = 0, ay = 0, az = 0, du = 0;
      int64_t c = 0;
      for (int64_t k = 0; k < b.n; ++k) {
        int64_t j = b.j[k];
        if (j == i) continue;
        ++c;
        double rr = b.r[k];
        if (rr == 0.0) continue;
        double dWi = (rr < h[i]) ? or_dWdr(rr, h[i]) : 0.0;
        double dWj = (rr < h[j]) ? or_dWdr(rr, h[j]) : 0.0;
        const double *d = b.d[k];
        double ex = d[0] / rr, ey = d[1] / rr, ez = d[2] / rr;
        double fac = m[j] * (A[i] * dWi + A[j] * dWj);
        ax -= fac * ex;
        ay -= fac * ey;
        az -= fac * ez;
        double dvx = v[3 * i] - v[3 * j], dvy = v[3 * i + 1] - v[3 * j + 1],
               dvz = v[3 * i + 2] - v[3 * j + 2];
        du += m[j] * dWi * (dvx * ex + dvy * ey + dvz * ez);
      }
      a[3 * i] = ax;
      a[3 * i + 1] = ay;
      a[3 * i + 2] = az;
      dudt[i] = A[i] * du;
      cnt[i] = c;
    }
    cand_free(&b);
  }
  if (use_tree) kd_free(&t);
  free(A);
  return rc;
}
