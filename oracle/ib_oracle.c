/*
 * ib_oracle.c -- FP64 reference for spreading and interpolation (arXiv 2012.06646).
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py, never by the CUDA library.
 * Compile with -ffp-contract=off so that X*(N/L) - xi is two rounded FP64 ops.
 */
#include "ib_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int g_mutation = 0;
void or_set_mutation(int m) { g_mutation = m; }

/* Kernels of Peskin (2002), cited by the paper in Section 2.
 * Standard 4-point: (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8 on |r| <= 1,
 *                   (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 on 1 <= |r| <= 2, else 0.
 * Cosine 4-point:   (1 + cos(pi r / 2))/4 on |r| <= 2, else 0.
 * Near |r| = 2 both definitions subtract nearly equal numbers.  They are
 * evaluated here in identical closed forms without that cancellation, so the
 * tail weights keep full relative accuracy:
 *   outer branch: multiply and divide by (5 - 2|r| + sqrt(...)); the
 *     numerator (5 - 2|r|)^2 - (-7 + 12|r| - 4r^2) equals 8 (2 - |r|)^2;
 *   cosine: 1 + cos(2 y) = 2 cos(y)^2 with y = pi r / 4. */
/* Kernels of other support widths (the methods of the paper do not depend on
 * phi, Section 2; s[phi] of Section 3.1 is 3 and 6 for these):
 * 3-point (Roma, Peskin and Berger 1999), s = 3:
 *   (1 + sqrt(1 - 3 r^2)) / 3                   on |r| <= 1/2,
 *   (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6    on 1/2 <= |r| <= 3/2, else 0;
 *   the outer branch is evaluated as (3 - 2|r|)^2 / (2 (5 - 3|r| + sqrt(...))),
 *   the same value without the cancellation near |r| = 3/2 (the numerator
 *   (5 - 3|r|)^2 - (1 - 3 (1 - |r|)^2) equals 3 (3 - 2|r|)^2).
 * 6-point B-spline (the centred quintic B-spline, six-fold convolution of the
 * unit box), s = 6, as its piecewise polynomial on |r| in [0,1), [1,2), [2,3):
 *   (66 - 60 r^2 + 30 r^4 - 10 |r|^5) / 120,
 *   (1 + 5c + 10c^2 + 10c^3 + 5c^4 - 5c^5) / 120 with c = 2 - |r|,
 *   (3 - |r|)^5 / 120, else 0;
 *   the middle piece is written in c = 2 - |r| so that it has no cancellation
 *   as |r| -> 2 (the same polynomial as the power form in |r|). */
static double phi_roma3(double r) {
  double a = fabs(r);
  if (a >= 1.5) return 0.0;
  if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
  double q = sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a));
  return (3.0 - 2.0 * a) * (3.0 - 2.0 * a) / (2.0 * (5.0 - 3.0 * a + q));
}

static double phi_bspline6(double r) {
  double a = fabs(r);
  if (a >= 3.0) return 0.0;
  if (a >= 2.0) {
    double c = 3.0 - a;
    return c * c * c * c * c / 120.0;
  }
  if (a >= 1.0) {
    double c = 2.0 - a;
    return (1.0 + 5.0 * c + 10.0 * c * c + 10.0 * c * c * c + 5.0 * c * c * c * c - 5.0 * c * c * c * c * c) / 120.0;
  }
  return (66.0 - 60.0 * a * a + 30.0 * a * a * a * a - 10.0 * a * a * a * a * a) / 120.0;
}

int or_width(int kernel) {
  if (kernel == 2) return 3;
  if (kernel == 3) return 6;
  return 4;
}

double or_phi(int kernel, double r) {
  if (kernel == 2) return phi_roma3(r);
  if (kernel == 3) return phi_bspline6(r);
  double a = fabs(r);
  if (a >= 2.0) return 0.0;
  if (kernel == 1) {
    /* cos(pi a / 4) = sin(pi (2 - a) / 4); 2 - a is exact for 1 <= a <= 2 */
    double c = (a < 1.0) ? cos(M_PI * a / 4.0) : sin(M_PI * (2.0 - a) / 4.0);
    return 0.5 * c * c;
  }
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  return (2.0 - a) * (2.0 - a) / (5.0 - 2.0 * a + sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
}

/* d phi / d r of the same formulas (both kernels are C^1 on the real line). */
/* Derivatives of the 3-point and 6-point kernels, from the same pieces:
 * 3-point: -r / sqrt(1 - 3 r^2) on |r| <= 1/2; sign(r) (-(1 + (1 - |r|) / q) / 2)
 *   with q = sqrt(1 - 3 (1 - |r|)^2) on 1/2 <= |r| <= 3/2 (0 at |r| = 3/2);
 * 6-point B-spline: sign(r) times (-120 a + 120 a^3 - 50 a^4) / 120 on [0, 1),
 *   -(5 + 20c + 30c^2 + 20c^3 - 25c^4) / 120 with c = 2 - a on [1, 2), and
 *   -(3 - a)^4 / 24 on [2, 3), a = |r|. */
static double dphi_roma3(double r) {
  double a = fabs(r), sgn = (r < 0.0) ? -1.0 : 1.0;
  if (a >= 1.5) return 0.0;
  if (a <= 0.5) return -r / sqrt(1.0 - 3.0 * r * r);
  double q = sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a));
  return sgn * (-(1.0 + (1.0 - a) / q) / 2.0);
}

static double dphi_bspline6(double r) {
  double a = fabs(r), sgn = (r < 0.0) ? -1.0 : 1.0;
  if (a >= 3.0) return 0.0;
  if (a >= 2.0) {
    double c = 3.0 - a;
    return sgn * (-(c * c * c * c) / 24.0);
  }
  if (a >= 1.0) {
    double c = 2.0 - a;
    return sgn * (-(5.0 + 20.0 * c + 30.0 * c * c + 20.0 * c * c * c - 25.0 * c * c * c * c) / 120.0);
  }
  return sgn * (-120.0 * a + 120.0 * a * a * a - 50.0 * a * a * a * a) / 120.0;
}

double or_dphi(int kernel, double r) {
  if (kernel == 2) return dphi_roma3(r);
  if (kernel == 3) return dphi_bspline6(r);
  double a = fabs(r);
  double sgn = (r < 0.0) ? -1.0 : 1.0;
  if (a >= 2.0) return 0.0;
  if (kernel == 1) return -(M_PI / 8.0) * sin(M_PI * r / 2.0);
  if (a <= 1.0) {
    double q = sqrt(1.0 + 4.0 * a - 4.0 * a * a);
    return sgn * (-2.0 + (2.0 - 4.0 * a) / q) / 8.0;
  }
  double q = sqrt(-7.0 + 12.0 * a - 4.0 * a * a);
  if (q == 0.0) return 0.0; /* |r| = 2 exactly is excluded above; guard the endpoint anyway */
  return sgn * (-2.0 - (6.0 - 4.0 * a) / q) / 8.0;
}

void or_cell(double X, double scale, double xi, long long* i, double* r) {
  volatile double u = X * scale; /* one rounded multiply */
  u = u - xi;                    /* one rounded subtract */
  double fl = floor(u);
  *i = (long long)fl;
  *r = u - fl;
}

double or_stagger(const or_grid* g, int comp, int b) {
  if (g->grid == 1) return (comp == b) ? 0.0 : 0.5;
  return 0.5;
}

static long long wrap(long long i, long long n) {
  long long m = i % n;
  return m < 0 ? m + n : m;
}

static long long ncell_of(const or_grid* g) {
  long long c = (long long)g->n[0] * g->n[1];
  if (g->dim == 3) c *= g->n[2];
  return c;
}

static int check_grid(const or_grid* g) {
  if (g->dim != 2 && g->dim != 3) return 1;
  for (int b = 0; b < g->dim; ++b)
    if (g->n[b] < 1 || !(g->L[b] > 0.0)) return 1;
  if (g->ncomp < 1) return 1;
  if (g->grid == 1 && g->ncomp != g->dim) return 1;
  if (g->kernel < 0 || g->kernel > 3) return 1;
  if (g->bounded & ~((1 << g->dim) - 1)) return 1;
  return 0;
}

int or_cell_keys(const or_grid* g, long long n, const double* X, unsigned long long* key) {
  if (check_grid(g)) return 1;
  for (long long j = 0; j < n; ++j) {
    unsigned long long k = 0, stride = 1;
    for (int b = 0; b < g->dim; ++b) {
      long long i;
      double r;
      or_cell(X[j * g->dim + b], (double)g->n[b] / g->L[b], 0.0, &i, &r);
      k += (unsigned long long)wrap(i, g->n[b]) * stride;
      stride *= (unsigned long long)g->n[b];
    }
    key[j] = k;
  }
  return 0;
}

long long or_bin_stable(long long n, const unsigned long long* key, unsigned long long nkeys,
                        long long* perm, long long* start) {
  long long* count = (long long*)calloc(nkeys + 1, sizeof(long long));
  long long q = 0;
  for (long long j = 0; j < n; ++j) count[key[j]] += 1;
  long long run = 0;
  for (unsigned long long k = 0; k < nkeys; ++k) {
    long long c = count[k];
    if (c > 0) ++q;
    start[k] = run;
    count[k] = run; /* next free slot of key k */
    run += c;
  }
  start[nkeys] = run;
  for (long long j = 0; j < n; ++j) perm[count[key[j]]++] = j; /* index order within a key: stable */
  free(count);
  return q;
}

/* Per point: cell index and offset for one component in every dimension. */
typedef struct {
  long long i[3];
  double r[3];
} cellrec;

static void point_cell(const or_grid* g, const double* Xj, int comp, cellrec* c) {
  for (int b = 0; b < g->dim; ++b) {
    or_cell(Xj[b], (double)g->n[b] / g->L[b], or_stagger(g, comp, b), &c->i[b], &c->r[b]);
  }
  if (g_mutation == 3 && g->dim >= 2) {
    double t = c->r[0];
    c->r[0] = c->r[1];
    c->r[1] = t;
  }
}

/* Nodes i + t examined around the cell i = floor(u) of a point, per
 * dimension: every node whose weight phi(t - r) can be nonzero for some
 * r in [0, 1), i.e. |t - r| < s/2.  Even s: t in [1 - s/2, s/2] (s nodes,
 * {-1, 0, 1, 2} for s = 4); odd s: t in [(1 - s)/2, (1 + s)/2] (s + 1 nodes,
 * one of which has weight 0 for any given r). */
static int window_lo(int kernel) {
  int s = or_width(kernel);
  return (s % 2 == 0) ? 1 - s / 2 : (1 - s) / 2;
}

static int window_n(int kernel) {
  int s = or_width(kernel);
  return (s % 2 == 0) ? s : s + 1;
}

static int nshift_of(const or_grid* g) {
  int w = window_n(g->kernel), m = 1;
  for (int b = 0; b < g->dim; ++b) m *= w;
  return m;
}

/* Shift number s (0-based) in colexicographic order, x fastest (Algorithm 1 with
 * the digits of s read base w, the window size), mapped to t = digit + window_lo. */
static void shift_of(const or_grid* g, int s, int* t) {
  int w = window_n(g->kernel), lo = window_lo(g->kernel);
  for (int b = 0; b < g->dim; ++b) {
    t[b] = (s % w) + lo;
    s /= w;
  }
}

/* Argument of phi for shift t and offset r: the displacement t - r of Eq. delta-defs. */
static double karg(int t, double r) { return (g_mutation == 2) ? (double)t + r : (double)t - r; }

/* Grid index of node i + t (periodic wrap), or -1 when it lies outside the
 * domain in a bounded dimension (the empty marker of the grid indexing function). */
static long long node_index(const or_grid* g, const cellrec* c, const int* t) {
  long long k = 0, stride = 1;
  for (int b = 0; b < g->dim; ++b) {
    long long i = c->i[b] + t[b];
    if ((g->bounded >> b) & 1) {
      if (i < 0 || i >= g->n[b]) return -1;
    } else {
      i = wrap(i, g->n[b]);
    }
    k += i * stride;
    stride *= g->n[b];
  }
  return k;
}

/* A point takes part only if it lies in [0, L_b] in every bounded dimension. */
static int point_in_domain(const or_grid* g, const double* Xj) {
  for (int b = 0; b < g->dim; ++b) {
    if (!((g->bounded >> b) & 1)) continue;
    volatile double u = Xj[b] * ((double)g->n[b] / g->L[b]);
    if (!(u >= 0.0 && u <= (double)g->n[b])) return 0;
  }
  return 1;
}

static double inv_cell_volume(const or_grid* g) {
  double v = 1.0;
  for (int b = 0; b < g->dim; ++b) v *= (double)g->n[b] / g->L[b];
  return v;
}

int or_spread(const or_grid* g, long long n, const double* X, const double* G, double* f, double* fabs_out) {
  if (check_grid(g)) return 1;
  long long ncell = ncell_of(g);
  int nshift = nshift_of(g);
  double hmd = (g_mutation == 1) ? 1.0 : inv_cell_volume(g);
  memset(f, 0, sizeof(double) * (size_t)(ncell * g->ncomp));
  if (fabs_out) memset(fabs_out, 0, sizeof(double) * (size_t)(ncell * g->ncomp));
  for (long long j = 0; j < n; ++j) {          /* loop over IB points (Algorithm 2) */
    if (!point_in_domain(g, X + j * g->dim)) continue;
    for (int a = 0; a < g->ncomp; ++a) {
      cellrec c;
      point_cell(g, X + j * g->dim, a, &c);
      for (int s = 0; s < nshift; ++s) {       /* loop over shifts */
        int t[3];
        shift_of(g, s, t);
        double w = 1.0;
        for (int b = 0; b < g->dim; ++b) w *= or_phi(g->kernel, karg(t[b], c.r[b]));
        long long k = node_index(g, &c, t);
        if (k < 0) continue;
        double contrib = hmd * w * G[j * g->ncomp + a];
        f[a * ncell + k] += contrib;
        if (fabs_out) fabs_out[a * ncell + k] += fabs(contrib);
      }
    }
  }
  return 0;
}

int or_interp(const or_grid* g, long long n, const double* X, const double* u, double* U, double* Uabs) {
  if (check_grid(g)) return 1;
  long long ncell = ncell_of(g);
  int nshift = nshift_of(g);
  for (long long j = 0; j < n; ++j) {          /* one independent row of S* per point (Algorithm 3) */
    if (!point_in_domain(g, X + j * g->dim)) {
      for (int a = 0; a < g->ncomp; ++a) {
        U[j * g->ncomp + a] = NAN;
        if (Uabs) Uabs[j * g->ncomp + a] = 0.0;
      }
      continue;
    }
    for (int a = 0; a < g->ncomp; ++a) {
      cellrec c;
      point_cell(g, X + j * g->dim, a, &c);
      double acc = 0.0, aabs = 0.0;
      for (int s = 0; s < nshift; ++s) {
        int t[3];
        shift_of(g, s, t);
        double w = 1.0;
        for (int b = 0; b < g->dim; ++b) w *= or_phi(g->kernel, karg(t[b], c.r[b]));
        long long k = node_index(g, &c, t);
        if (k < 0) continue;
        double term = w * u[a * ncell + k];
        acc += term;
        aabs += fabs(term);
      }
      U[j * g->ncomp + a] = acc;
      if (Uabs) Uabs[j * g->ncomp + a] = aabs;
    }
  }
  return 0;
}

int or_pos_grad(const or_grid* g, long long n, const double* X, const double* field, const double* v,
                double* D, double* Dabs) {
  if (check_grid(g)) return 1;
  long long ncell = ncell_of(g);
  int nshift = nshift_of(g);
  for (long long j = 0; j < n; ++j) {
    if (!point_in_domain(g, X + j * g->dim)) {   /* outside a bounded dimension: no gradient */
      for (int b = 0; b < g->dim; ++b) {
        D[j * g->dim + b] = NAN;
        if (Dabs) Dabs[j * g->dim + b] = 0.0;
      }
      continue;
    }
    for (int b = 0; b < g->dim; ++b) {
      double acc = 0.0, aabs = 0.0;
      /* d r_b / d X_b = N_b / L_b, and the weight depends on r_b through phi(t_b - r_b). */
      double drdx = (double)g->n[b] / g->L[b];
      double chain = (g_mutation == 4) ? drdx : -drdx;
      for (int a = 0; a < g->ncomp; ++a) {
        cellrec c;
        point_cell(g, X + j * g->dim, a, &c);
        for (int s = 0; s < nshift; ++s) {
          int t[3];
          shift_of(g, s, t);
          double w = chain * or_dphi(g->kernel, karg(t[b], c.r[b]));
          for (int e = 0; e < g->dim; ++e)
            if (e != b) w *= or_phi(g->kernel, karg(t[e], c.r[e]));
          long long k = node_index(g, &c, t);
          if (k < 0) continue;
          double term = v[j * g->ncomp + a] * w * field[a * ncell + k];
          acc += term;
          aabs += fabs(term);
        }
      }
      D[j * g->dim + b] = acc;
      if (Dabs) Dabs[j * g->dim + b] = aabs;
    }
  }
  return 0;
}
