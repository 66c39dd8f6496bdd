/*
 * FP64 CPU oracle for the compressed DP-SE_a path -- TEST INFRASTRUCTURE.
 * Only the tests, the smoke check and the CPU-baseline leg of the bench call
 * this library.  It is deliberately plain: one atom at a time, no blocking,
 * no fusion, every intermediate in float64.  See oracle.h for the passages
 * each function follows.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXT 8
#define MAXL 8

struct orc_model {
  int ntypes, n_emb, emb_w[MAXL], m_lt, n_fit, fit_w[MAXL];
  int M, din;
  const double* emb_W[MAXT * MAXT][MAXL];
  const double* emb_b[MAXT * MAXT][MAXL];
  const double* fit_W[MAXT][MAXL];
  const double* fit_b[MAXT][MAXL];
  const double* fit_wout[MAXT];
  double fit_bout[MAXT];
  double* data;
};

struct orc_table {
  int ntypes, M, n;
  double h;
  int n_fine; /* intervals of width h on [0, n_fine h]; the rest, up to n, */
  double H;   /* of width H (the extrapolation region; n_fine = n without) */
  double* a;  /* [ntypes*ntypes][n][6][M] */
};

/* node k of the table: k h in the first region, n_fine h + (k - n_fine) H
 * beyond it */
static double tab_node(const orc_table* t, int k) {
  return k <= t->n_fine ? k * t->h : t->n_fine * t->h + (k - t->n_fine) * t->H;
}

static double tab_width(const orc_table* t, int k) { return k < t->n_fine ? t->h : t->H; }

/* interval k owning s (interval k is [x_k, x_{k+1}), clamped to the table)
 * and the local variable s - x_k */
static double tab_locate(const orc_table* t, double s, int* k_out) {
  const double s_fine = t->n_fine * t->h;
  double fk;
  int k;
  if (s < s_fine || t->n == t->n_fine) {
    fk = floor(s / t->h);
    k = fk < 0 ? 0 : (fk > t->n_fine - 1 ? t->n_fine - 1 : (int)fk);
  } else {
    fk = floor((s - s_fine) / t->H);
    const int last = t->n - t->n_fine - 1;
    k = t->n_fine + (fk < 0 ? 0 : (fk > last ? last : (int)fk));
  }
  *k_out = k;
  return s - tab_node(t, k);
}

void orc_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* model file                                                                */
/* ------------------------------------------------------------------------ */
orc_model* orc_model_load(const char* path) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  char magic[8];
  orc_model* m = NULL;
  int32_t buf[64];
  int nint = 0;
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "DPSEAV01", 8) != 0) goto fail;
  m = (orc_model*)calloc(1, sizeof(orc_model));
  if (!m) goto fail;
  if (fread(buf, 4, 2, f) != 2) goto fail;
  m->ntypes = buf[0];
  m->n_emb = buf[1];
  nint = 2;
  if (m->ntypes < 1 || m->ntypes > MAXT || m->n_emb < 1 || m->n_emb > MAXL) goto fail;
  if (fread(m->emb_w, 4, (size_t)m->n_emb, f) != (size_t)m->n_emb) goto fail;
  nint += m->n_emb;
  if (fread(buf, 4, 2, f) != 2) goto fail;
  m->m_lt = buf[0];
  m->n_fit = buf[1];
  nint += 2;
  if (m->n_fit < 1 || m->n_fit > MAXL - 1) goto fail;
  if (fread(m->fit_w, 4, (size_t)m->n_fit, f) != (size_t)m->n_fit) goto fail;
  nint += m->n_fit;
  if (nint % 2) {
    if (fread(buf, 4, 1, f) != 1) goto fail;
  }
  for (int k = 1; k < m->n_emb; ++k)
    if (m->emb_w[k] != 2 * m->emb_w[k - 1]) goto fail; /* Eq. 5 doubles the width */
  m->M = m->emb_w[m->n_emb - 1];
  if (m->m_lt < 1 || m->m_lt > m->M) goto fail;
  m->din = m->M * m->m_lt;
  /* count doubles */
  size_t total = 0;
  int np = m->ntypes * m->ntypes;
  for (int p = 0; p < np; ++p) {
    int prev = 1;
    for (int k = 0; k < m->n_emb; ++k) {
      total += (size_t)prev * m->emb_w[k] + m->emb_w[k];
      prev = m->emb_w[k];
    }
  }
  for (int t = 0; t < m->ntypes; ++t) {
    int prev = m->din;
    for (int k = 0; k < m->n_fit; ++k) {
      total += (size_t)prev * m->fit_w[k] + m->fit_w[k];
      prev = m->fit_w[k];
    }
    total += (size_t)prev + 1;
  }
  m->data = (double*)malloc(total * sizeof(double));
  if (!m->data) goto fail;
  if (fread(m->data, sizeof(double), total, f) != total) goto fail;
  {
    char extra;
    if (fread(&extra, 1, 1, f) != 0) goto fail; /* trailing bytes: malformed */
  }
  fclose(f);
  f = NULL;
  double* q = m->data;
  for (int p = 0; p < np; ++p) {
    int prev = 1;
    for (int k = 0; k < m->n_emb; ++k) {
      m->emb_W[p][k] = q;
      q += (size_t)prev * m->emb_w[k];
      m->emb_b[p][k] = q;
      q += m->emb_w[k];
      prev = m->emb_w[k];
    }
  }
  for (int t = 0; t < m->ntypes; ++t) {
    int prev = m->din;
    for (int k = 0; k < m->n_fit; ++k) {
      m->fit_W[t][k] = q;
      q += (size_t)prev * m->fit_w[k];
      m->fit_b[t][k] = q;
      q += m->fit_w[k];
      prev = m->fit_w[k];
    }
    m->fit_wout[t] = q;
    q += prev;
    m->fit_bout[t] = *q;
    q += 1;
  }
  return m;
fail:
  if (f) fclose(f);
  if (m) {
    free(m->data);
    free(m);
  }
  return NULL;
}

void orc_model_free(orc_model* m) {
  if (!m) return;
  free(m->data);
  free(m);
}

int orc_model_dims(const orc_model* m, int32_t* dims) {
  if (!m || !dims) return ORC_ERR_ARG;
  dims[0] = m->ntypes;
  dims[1] = m->M;
  dims[2] = m->m_lt;
  dims[3] = m->din;
  dims[4] = m->emb_w[0];
  dims[5] = m->n_fit;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: switch and environment-matrix row                                   */
/* ------------------------------------------------------------------------ */
void orc_switch(double r, double rc, double rcs, double* sw, double* dsw) {
  if (r < rcs) {
    *sw = 1.0;
    *dsw = 0.0;
  } else if (r < rc) {
    double w = rc - rcs;
    double u = (r - rcs) / w;
    double u2 = u * u, u3 = u2 * u;
    *sw = 1.0 - 10.0 * u3 + 15.0 * u3 * u - 6.0 * u3 * u2;
    *dsw = (-30.0 * u2 + 60.0 * u3 - 30.0 * u3 * u) / w;
  } else {
    *sw = 0.0;
    *dsw = 0.0;
  }
}

double orc_env_row(const double* d, double rc, double rcs, double* R, double* dR) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double r = sqrt(r2);
  double sw, dsw;
  orc_switch(r, rc, rcs, &sw, &dsw);
  double s = sw / r;
  double ds = dsw / r - sw / r2; /* ds/dr */
  double u[3] = {d[0] / r, d[1] / r, d[2] / r};
  R[0] = s;
  for (int a = 0; a < 3; ++a) R[1 + a] = s * u[a];
  if (dR) {
    /* dR_0/dd_b = s' u_b ; dR_{1+a}/dd_b = s' u_a u_b + (s/r)(delta_ab - u_a u_b) */
    for (int b = 0; b < 3; ++b) dR[0 * 3 + b] = ds * u[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        dR[(1 + a) * 3 + b] = ds * u[a] * u[b] + (s / r) * ((a == b ? 1.0 : 0.0) - u[a] * u[b]);
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3-5: embedding net with forward-mode first and second derivatives      */
/* ------------------------------------------------------------------------ */
int orc_embed(const orc_model* m, int ti, int tj, double s, double* g, double* dg, double* d2g) {
  if (!m || ti < 0 || tj < 0 || ti >= m->ntypes || tj >= m->ntypes) return ORC_ERR_ARG;
  int p = ti * m->ntypes + tj;
  int wmax = m->M;
  double* h = (double*)malloc(sizeof(double) * 6 * (size_t)wmax);
  if (!h) return ORC_ERR_NOMEM;
  double *h1 = h + wmax, *h2 = h + 2 * wmax; /* value, 1st, 2nd derivative */
  double *o0 = h + 3 * wmax, *o1 = h + 4 * wmax, *o2 = h + 5 * wmax;
  /* layer 0: tanh(s W0 + b0) (Eq. 4) */
  int w = m->emb_w[0];
  for (int k = 0; k < w; ++k) {
    double z = s * m->emb_W[p][0][k] + m->emb_b[p][0][k];
    double zp = m->emb_W[p][0][k];
    double t = tanh(z);
    double q = 1.0 - t * t;
    h[k] = t;
    h1[k] = q * zp;
    h2[k] = -2.0 * t * q * zp * zp;
  }
  /* layers k>=1: (x,x) + tanh(x W + b) (Eq. 5) */
  for (int L = 1; L < m->n_emb; ++L) {
    int wo = m->emb_w[L];
    const double* W = m->emb_W[p][L];
    const double* b = m->emb_b[p][L];
    for (int c = 0; c < wo; ++c) {
      double z = b[c], zp = 0.0, zpp = 0.0;
      for (int k = 0; k < w; ++k) {
        double wk = W[(size_t)k * wo + c];
        z += h[k] * wk;
        zp += h1[k] * wk;
        zpp += h2[k] * wk;
      }
      double t = tanh(z);
      double q = 1.0 - t * t;
      int src = c % w; /* (x,x): output column c repeats input column c mod w */
      o0[c] = h[src] + t;
      o1[c] = h1[src] + q * zp;
      o2[c] = h2[src] + q * zpp - 2.0 * t * q * zp * zp;
    }
    memcpy(h, o0, sizeof(double) * wo);
    memcpy(h1, o1, sizeof(double) * wo);
    memcpy(h2, o2, sizeof(double) * wo);
    w = wo;
  }
  memcpy(g, h, sizeof(double) * w);
  if (dg) memcpy(dg, h1, sizeof(double) * w);
  if (d2g) memcpy(d2g, h2, sizeof(double) * w);
  free(h);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5: tanh of the fitting net tabulated on [0, 8) by a second-order    */
/* polynomial per interval, odd symmetry, 1 for |x| >= 8.  Reading (the paper */
/* fixes neither the step nor the conditions): step h = 1/128; on             */
/* [x_k, x_k + h], p(u) = a0 + a1 u + a2 u^2 with p(0) = tanh(x_k),           */
/* p'(0) = 1 - tanh(x_k)^2 and p(h) = tanh(x_k + h).  The derivative used in  */
/* the gradient is p'(u), so forces stay the gradient of the computed energy. */
/* ------------------------------------------------------------------------ */
#define TT_N 1024
#define TT_PER_UNIT 128.0
static int g_tanh_table = 0;
static int g_tt_ready = 0;
static double g_tt[TT_N][3];

void orc_set_tanh_table(int on) {
  if (on && !g_tt_ready) {
    const double h = 1.0 / TT_PER_UNIT;
    for (int k = 0; k < TT_N; ++k) {
      const double x0 = k * h;
      const double y0 = tanh(x0), y1 = tanh(x0 + h);
      g_tt[k][0] = y0;
      g_tt[k][1] = 1.0 - y0 * y0;
      g_tt[k][2] = (y1 - g_tt[k][0] - g_tt[k][1] * h) / (h * h);
    }
    g_tt_ready = 1;
  }
  g_tanh_table = on ? 1 : 0;
}

/* the fitting net's activation: t = tanh(a) (or its table), dt = dt/da */
double orc_act(double a, double* dt) {
  if (!g_tanh_table) {
    const double t = tanh(a);
    if (dt) *dt = 1.0 - t * t;
    return t;
  }
  const double ax = fabs(a);
  if (ax >= 8.0) {
    if (dt) *dt = 0.0;
    return a > 0 ? 1.0 : -1.0;
  }
  int k = (int)(ax * TT_PER_UNIT);
  if (k > TT_N - 1) k = TT_N - 1;
  const double u = ax - k / TT_PER_UNIT;
  const double p = g_tt[k][0] + u * (g_tt[k][1] + u * g_tt[k][2]);
  if (dt) *dt = g_tt[k][1] + 2.0 * g_tt[k][2] * u;
  return a < 0 ? -p : p;
}

/* ------------------------------------------------------------------------ */
/* fitting net (Sec. 2.1): hidden layers tanh, shortcut on equal widths       */
/* ------------------------------------------------------------------------ */
int orc_fit(const orc_model* m, int ti, const double* D, double* E, double* dD) {
  if (!m || ti < 0 || ti >= m->ntypes) return ORC_ERR_ARG;
  int nf = m->n_fit;
  size_t tot = 0;
  for (int k = 0; k < nf; ++k) tot += (size_t)m->fit_w[k];
  double* z = (double*)malloc(sizeof(double) * (2 * tot + 2 * (size_t)m->din + 16));
  if (!z) return ORC_ERR_NOMEM;
  double* tk = z + tot; /* activation derivatives per layer */
  size_t off[MAXL + 1];
  off[0] = 0;
  for (int k = 0; k < nf; ++k) off[k + 1] = off[k] + (size_t)m->fit_w[k];
  const double* in = D;
  int win = m->din;
  for (int k = 0; k < nf; ++k) {
    int wo = m->fit_w[k];
    const double* W = m->fit_W[ti][k];
    const double* b = m->fit_b[ti][k];
    int shortcut = (k > 0 && wo == win);
    for (int c = 0; c < wo; ++c) {
      double a = b[c];
      for (int r = 0; r < win; ++r) a += in[r] * W[(size_t)r * wo + c];
      double dt;
      const double t = orc_act(a, &dt);
      tk[off[k] + c] = dt;
      z[off[k] + c] = (shortcut ? in[c] : 0.0) + t;
    }
    in = z + off[k];
    win = wo;
  }
  double e = m->fit_bout[ti];
  for (int c = 0; c < win; ++c) e += in[c] * m->fit_wout[ti][c];
  *E = e;
  if (dD) {
    double* gz = z + 2 * tot;          /* gradient wrt current layer output */
    double* gn = gz + m->din;          /* gradient wrt previous output */
    for (int c = 0; c < win; ++c) gz[c] = m->fit_wout[ti][c];
    for (int k = nf - 1; k >= 0; --k) {
      int wo = m->fit_w[k];
      int wi = (k == 0) ? m->din : m->fit_w[k - 1];
      int shortcut = (k > 0 && wo == wi);
      const double* W = m->fit_W[ti][k];
      for (int r = 0; r < wi; ++r) gn[r] = 0.0;
      for (int c = 0; c < wo; ++c) {
        double gp = gz[c] * tk[off[k] + c]; /* through the activation */
        for (int r = 0; r < wi; ++r) gn[r] += W[(size_t)r * wo + c] * gp;
        if (shortcut) gn[c] += gz[c];
      }
      double* sw = gz;
      gz = gn;
      gn = sw;
    }
    memcpy(dD, gz, sizeof(double) * m->din);
  }
  free(z);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2 tabulation                                                       */
/* ------------------------------------------------------------------------ */
void orc_hermite5(const double* y0, const double* y1, double h, double* a) {
  /* f(t)=sum a_k t^k on [0,h]; f,f',f'' match (y0) at t=0 and (y1) at t=h.
   * The t=0 conditions give a0..a2 directly.  With p=a3 h^3, q=a4 h^4,
   * w=a5 h^5 the t=h conditions read
   *   p +  q +  w = A            A = y1 - y0 - y0' h - y0'' h^2/2
   *  3p + 4q + 5w = B h          B = y1' - y0' - y0'' h
   *  6p +12q +20w = C h^2        C = y1'' - y0''
   * whose solution is p = 10A - 4Bh + Ch^2/2, q = -15A + 7Bh - Ch^2,
   * w = 6A - 3Bh + Ch^2/2. */
  double A = y1[0] - y0[0] - y0[1] * h - 0.5 * y0[2] * h * h;
  double B = y1[1] - y0[1] - y0[2] * h;
  double C = y1[2] - y0[2];
  double h2 = h * h, h3 = h2 * h;
  a[0] = y0[0];
  a[1] = y0[1];
  a[2] = 0.5 * y0[2];
  a[3] = (10.0 * A - 4.0 * B * h + 0.5 * C * h2) / h3;
  a[4] = (-15.0 * A + 7.0 * B * h - C * h2) / (h3 * h);
  a[5] = (6.0 * A - 3.0 * B * h + 0.5 * C * h2) / (h3 * h2);
}

orc_table* orc_table_build(const orc_model* m, double h, double s_max) {
  return orc_table_build_ext(m, h, s_max, 0.0, 1);
}

orc_table* orc_table_build_ext(const orc_model* m, double h, double s_max, double s_ext,
                               int stride) {
  if (!m || !(h > 0) || !(s_max > 0) || stride < 1) return NULL;
  int n_fine = (int)ceil(s_max / h - 1e-9);
  if (n_fine < 1) n_fine = 1;
  const double H = stride * h;
  const double rest = s_ext - n_fine * h;
  const int n_ext = rest > 0 ? (int)ceil(rest / H - 1e-9) : 0;
  const int n = n_fine + (n_ext > 0 ? n_ext : 0);
  orc_table* t = (orc_table*)calloc(1, sizeof(orc_table));
  if (!t) return NULL;
  t->ntypes = m->ntypes;
  t->M = m->M;
  t->n = n;
  t->h = h;
  t->n_fine = n_fine;
  t->H = H;
  int np = m->ntypes * m->ntypes, M = m->M;
  t->a = (double*)malloc(sizeof(double) * (size_t)np * n * 6 * M);
  double* node = (double*)malloc(sizeof(double) * (size_t)np * (n + 1) * 3 * M);
  if (!t->a || !node) {
    free(t->a);
    free(node);
    free(t);
    return NULL;
  }
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int idx = 0; idx < np * (n + 1); ++idx) {
    int p = idx / (n + 1), k = idx % (n + 1);
    double* nd = node + (size_t)idx * 3 * M;
    err |= orc_embed(m, p / m->ntypes, p % m->ntypes, tab_node(t, k), nd, nd + M, nd + 2 * M);
  }
  if (err) {
    free(node);
    orc_table_free(t);
    return NULL;
  }
  for (int p = 0; p < np; ++p)
    for (int k = 0; k < n; ++k) {
      const double* n0 = node + ((size_t)p * (n + 1) + k) * 3 * M;
      const double* n1 = n0 + 3 * M;
      for (int c = 0; c < M; ++c) {
        double y0[3] = {n0[c], n0[M + c], n0[2 * M + c]};
        double y1[3] = {n1[c], n1[M + c], n1[2 * M + c]};
        double a[6];
        orc_hermite5(y0, y1, tab_width(t, k), a);
        for (int q = 0; q < 6; ++q) t->a[(((size_t)p * n + k) * 6 + q) * M + c] = a[q];
      }
    }
  free(node);
  return t;
}

void orc_table_free(orc_table* t) {
  if (!t) return;
  free(t->a);
  free(t);
}

int orc_table_dims(const orc_table* t, int32_t* n, double* h) {
  if (!t) return ORC_ERR_ARG;
  if (n) *n = t->n;
  if (h) *h = t->h;
  return ORC_OK;
}

int orc_table_ext(const orc_table* t, int32_t* n_fine, double* H) {
  if (!t) return ORC_ERR_ARG;
  if (n_fine) *n_fine = t->n_fine;
  if (H) *H = t->H;
  return ORC_OK;
}

int orc_table_coeffs(const orc_table* t, int ti, int tj, double* out) {
  if (!t || ti < 0 || tj < 0 || ti >= t->ntypes || tj >= t->ntypes) return ORC_ERR_ARG;
  size_t sz = (size_t)t->n * 6 * t->M;
  memcpy(out, t->a + (size_t)(ti * t->ntypes + tj) * sz, sizeof(double) * sz);
  return ORC_OK;
}

int orc_table_eval(const orc_table* t, int ti, int tj, double s, double* g, double* dg) {
  /* interval k owns [x_k, x_{k+1}); local variable u = s - x_k (a reading:
   * the paper writes global powers of x, which is the same polynomial).
   * s = sw(r)/r >= 0; a rounding-level negative s next to rc evaluates the
   * first interval, so only s beyond the last node is out of range */
  int out = (s > tab_node(t, t->n)) ? 1 : 0;
  int k;
  double u = tab_locate(t, s, &k);
  int M = t->M;
  const double* a = t->a + ((size_t)(ti * t->ntypes + tj) * t->n + k) * 6 * M;
  for (int c = 0; c < M; ++c) {
    double a0 = a[c], a1 = a[M + c], a2 = a[2 * M + c], a3 = a[3 * M + c], a4 = a[4 * M + c],
           a5 = a[5 * M + c];
    g[c] = a0 + u * (a1 + u * (a2 + u * (a3 + u * (a4 + u * a5))));
    if (dg) dg[c] = a1 + u * (2.0 * a2 + u * (3.0 * a3 + u * (4.0 * a4 + u * 5.0 * a5)));
  }
  return out;
}

/* ------------------------------------------------------------------------ */
/* neighbors                                                                 */
/* ------------------------------------------------------------------------ */
double orc_wrap(double x, double L) {
  double w = x - floor(x / L) * L;
  if (w >= L) w -= L;
  if (w < 0.0) w += L;
  return w;
}

typedef struct {
  int64_t n;
  double L[3];
  int nc[3];
  int64_t* head; /* [ncell+1] CSR start */
  int64_t* atoms;
  double* xw; /* wrapped positions [n][3] */
} cells_t;

static int box_lengths(const double* box, double* L) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && box[a * 3 + b] != 0.0) return ORC_ERR_BOX; /* orthorhombic only */
  for (int a = 0; a < 3; ++a) {
    L[a] = box[a * 4];
    if (!(L[a] > 0)) return ORC_ERR_BOX;
  }
  return ORC_OK;
}

static int cells_build(cells_t* c, int64_t n, const double* x, const double* L, double rlist) {
  memset(c, 0, sizeof(*c));
  c->n = n;
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    c->L[a] = L[a];
    if (L[a] < rlist) return ORC_ERR_BOX; /* images |n|>=2 would be needed */
    c->nc[a] = (int)floor(L[a] / rlist);
    if (c->nc[a] < 1) c->nc[a] = 1;
    ncell *= c->nc[a];
  }
  c->xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  c->head = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  c->atoms = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!c->xw || !c->head || !c->atoms || !cid) {
    free(cid);
    return ORC_ERR_NOMEM;
  }
  for (int64_t i = 0; i < n; ++i) {
    int ci[3];
    for (int a = 0; a < 3; ++a) {
      double w = orc_wrap(x[i * 3 + a], L[a]);
      c->xw[i * 3 + a] = w;
      ci[a] = (int)floor(w / L[a] * c->nc[a]);
      if (ci[a] >= c->nc[a]) ci[a] = c->nc[a] - 1;
      if (ci[a] < 0) ci[a] = 0;
    }
    cid[i] = ((int64_t)ci[0] * c->nc[1] + ci[1]) * c->nc[2] + ci[2];
    c->head[cid[i] + 1]++;
  }
  for (int64_t k = 0; k < ncell; ++k) c->head[k + 1] += c->head[k];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  if (!fill) {
    free(cid);
    return ORC_ERR_NOMEM;
  }
  memcpy(fill, c->head, sizeof(int64_t) * (size_t)ncell);
  for (int64_t i = 0; i < n; ++i) c->atoms[fill[cid[i]]++] = i; /* ascending i per cell */
  free(fill);
  free(cid);
  return ORC_OK;
}

static void cells_free(cells_t* c) {
  free(c->xw);
  free(c->head);
  free(c->atoms);
}

typedef struct {
  int64_t j;
  int img[3];
  double d[3];
} nbr_t;

/* all (j,n) within rlist of atom i, via the cell list (27-cell stencil; each
 * stencil offset carries its own periodic image, so visiting one cell twice
 * with different images is correct when a box edge holds fewer than 3 cells) */
static int64_t cells_neighbors(const cells_t* c, int64_t i, double rlist, nbr_t* out, int64_t cap) {
  double r2max = rlist * rlist;
  const double* xi = c->xw + i * 3;
  int ci[3];
  for (int a = 0; a < 3; ++a) {
    ci[a] = (int)floor(xi[a] / c->L[a] * c->nc[a]);
    if (ci[a] >= c->nc[a]) ci[a] = c->nc[a] - 1;
    if (ci[a] < 0) ci[a] = 0;
  }
  int64_t cnt = 0;
  for (int ox = -1; ox <= 1; ++ox)
    for (int oy = -1; oy <= 1; ++oy)
      for (int oz = -1; oz <= 1; ++oz) {
        int o[3] = {ox, oy, oz}, cc[3], img[3];
        for (int a = 0; a < 3; ++a) {
          int v = ci[a] + o[a];
          img[a] = (v < 0) ? -1 : (v >= c->nc[a] ? 1 : 0);
          cc[a] = v - img[a] * c->nc[a];
        }
        int64_t cell = ((int64_t)cc[0] * c->nc[1] + cc[1]) * c->nc[2] + cc[2];
        for (int64_t q = c->head[cell]; q < c->head[cell + 1]; ++q) {
          int64_t j = c->atoms[q];
          if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
          double d[3], r2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            d[a] = (c->xw[j * 3 + a] - xi[a]) + img[a] * c->L[a];
            r2 += d[a] * d[a];
          }
          if (r2 < r2max) {
            if (cnt < cap) {
              out[cnt].j = j;
              for (int a = 0; a < 3; ++a) {
                out[cnt].img[a] = img[a];
                out[cnt].d[a] = d[a];
              }
            }
            cnt++;
          }
        }
      }
  return cnt;
}

static int cmp5(const void* pa, const void* pb) {
  const int32_t *a = (const int32_t*)pa, *b = (const int32_t*)pb;
  for (int k = 0; k < 5; ++k)
    if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
  return 0;
}

int64_t orc_neighbors(int64_t n, const double* x, const double* box, double rlist, int method,
                      int64_t cap, int32_t* out5) {
  double L[3];
  if (box_lengths(box, L) != ORC_OK) return -ORC_ERR_BOX;
  if (!(rlist > 0)) return -ORC_ERR_ARG;
  int64_t cnt = 0;
  if (method == 0) {
    double* xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!xw) return -ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n * 3; ++i) xw[i] = orc_wrap(x[i], L[i % 3]);
    int nm[3];
    for (int a = 0; a < 3; ++a) nm[a] = (int)ceil(rlist / L[a]) + 1;
    double r2max = rlist * rlist;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        for (int nx = -nm[0]; nx <= nm[0]; ++nx)
          for (int ny = -nm[1]; ny <= nm[1]; ++ny)
            for (int nz = -nm[2]; nz <= nm[2]; ++nz) {
              if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
              int img[3] = {nx, ny, nz};
              double r2 = 0.0;
              for (int a = 0; a < 3; ++a) {
                double d = (xw[j * 3 + a] - xw[i * 3 + a]) + img[a] * L[a];
                r2 += d * d;
              }
              if (r2 < r2max) {
                if (cnt < cap) {
                  int32_t* o = out5 + cnt * 5;
                  o[0] = (int32_t)i;
                  o[1] = (int32_t)j;
                  o[2] = nx;
                  o[3] = ny;
                  o[4] = nz;
                }
                cnt++;
              }
            }
    free(xw);
  } else {
    cells_t c;
    int e = cells_build(&c, n, x, L, rlist);
    if (e != ORC_OK) {
      cells_free(&c);
      return -e;
    }
    nbr_t* buf = NULL;
    int64_t bcap = 0;
    for (int64_t i = 0; i < n; ++i) {
      int64_t k = cells_neighbors(&c, i, rlist, buf, bcap);
      if (k > bcap) {
        free(buf);
        bcap = 2 * k;
        buf = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)bcap);
        if (!buf) {
          cells_free(&c);
          return -ORC_ERR_NOMEM;
        }
        k = cells_neighbors(&c, i, rlist, buf, bcap);
      }
      for (int64_t q = 0; q < k; ++q) {
        if (cnt < cap) {
          int32_t* o = out5 + cnt * 5;
          o[0] = (int32_t)i;
          o[1] = (int32_t)buf[q].j;
          o[2] = buf[q].img[0];
          o[3] = buf[q].img[1];
          o[4] = buf[q].img[2];
        }
        cnt++;
      }
    }
    free(buf);
    cells_free(&c);
  }
  if (cnt <= cap && out5) qsort(out5, (size_t)cnt, 5 * sizeof(int32_t), cmp5);
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* per-atom evaluation                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_model* m;
  const orc_table* tab;
  double rc, rcs;
  const int32_t* sel;
  int Nm; /* sum of sel: the N_m of Eq. 2 */
  const int32_t* types;
  const cells_t* cells;
} ctx_t;

typedef struct {
  nbr_t* nb;
  int64_t cap;
  double* G;  /* [cap][M] */
  double* dG; /* [cap][M] */
  double* R;  /* [cap][4] */
  double* dR; /* [cap][12] */
  double *T, *D, *dD, *dT;
} work_t;

static int work_init(work_t* w, const orc_model* m, int64_t cap) {
  memset(w, 0, sizeof(*w));
  w->cap = cap;
  int M = m->M;
  w->nb = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)cap);
  w->G = (double*)malloc(sizeof(double) * (size_t)cap * M);
  w->dG = (double*)malloc(sizeof(double) * (size_t)cap * M);
  w->R = (double*)malloc(sizeof(double) * (size_t)cap * 4);
  w->dR = (double*)malloc(sizeof(double) * (size_t)cap * 12);
  w->T = (double*)malloc(sizeof(double) * 4 * (size_t)M);
  w->dT = (double*)malloc(sizeof(double) * 4 * (size_t)M);
  w->D = (double*)malloc(sizeof(double) * (size_t)m->din);
  w->dD = (double*)malloc(sizeof(double) * (size_t)m->din);
  return (w->nb && w->G && w->dG && w->R && w->dR && w->T && w->dT && w->D && w->dD)
             ? ORC_OK
             : ORC_ERR_NOMEM;
}

static void work_free(work_t* w) {
  free(w->nb);
  free(w->G);
  free(w->dG);
  free(w->R);
  free(w->dR);
  free(w->T);
  free(w->dT);
  free(w->D);
  free(w->dD);
}

/* Energy of atom i and, when g_out != NULL, g_ij = dE_i/dr_ij for every
 * neighbor (written in the order of w->nb).  Returns the neighbor count in
 * *nnb.  flags: bit0 sel overflow, bit1 table range. */
static int atom_eval(const ctx_t* C, int64_t i, work_t* w, double* Ei, double* g_out,
                     int64_t* nnb, int* flags) {
  const orc_model* m = C->m;
  int M = m->M, mlt = m->m_lt, ti = C->types[i];
  int64_t k = cells_neighbors(C->cells, i, C->rc, w->nb, w->cap);
  if (k > w->cap) return ORC_ERR_SEL; /* beyond any sel: caller sized cap generously */
  *nnb = k;
  int cnt_t[MAXT] = {0};
  for (int64_t q = 0; q < k; ++q) cnt_t[C->types[w->nb[q].j]]++;
  for (int t = 0; t < m->ntypes; ++t)
    if (cnt_t[t] > C->sel[t]) *flags |= 1;
  double inv_nm = 1.0 / (double)C->Nm; /* reading: T = R^T G / N_m */
  for (int c = 0; c < 4 * M; ++c) w->T[c] = 0.0;
  for (int64_t q = 0; q < k; ++q) {
    int tj = C->types[w->nb[q].j];
    double* R = w->R + q * 4;
    double s = orc_env_row(w->nb[q].d, C->rc, C->rcs, R, w->dR + q * 12);
    double* G = w->G + q * M;
    double* dG = w->dG + q * M;
    if (C->tab) {
      if (orc_table_eval(C->tab, ti, tj, s, G, dG)) *flags |= 2;
    } else {
      orc_embed(m, ti, tj, s, G, dG, NULL);
    }
    for (int c = 0; c < 4; ++c)
      for (int e = 0; e < M; ++e) w->T[c * M + e] += R[c] * G[e] * inv_nm;
  }
  /* Eq. 2 with the reading D[b*m_lt + a] = sum_c T[c][b] T[c][a], a < M^< */
  for (int b = 0; b < M; ++b)
    for (int a = 0; a < mlt; ++a) {
      double s = 0.0;
      for (int c = 0; c < 4; ++c) s += w->T[c * M + b] * w->T[c * M + a];
      w->D[b * mlt + a] = s;
    }
  int e = orc_fit(m, ti, w->D, Ei, g_out ? w->dD : NULL);
  if (e) return e;
  if (!g_out) return ORC_OK;
  /* dE/dT from dE/dD (both factors of Eq. 2) */
  for (int c = 0; c < 4; ++c)
    for (int x = 0; x < M; ++x) {
      double s = 0.0;
      for (int a = 0; a < mlt; ++a) s += w->dD[x * mlt + a] * w->T[c * M + a];
      if (x < mlt)
        for (int b = 0; b < M; ++b) s += w->dD[b * mlt + x] * w->T[c * M + b];
      w->dT[c * M + x] = s;
    }
  /* back through T = (1/N_m) sum_j R_j^T g(s_j) and Eq. 1 to r_ij */
  for (int64_t q = 0; q < k; ++q) {
    const double* R = w->R + q * 4;
    const double* dR = w->dR + q * 12;
    const double* G = w->G + q * M;
    const double* dG = w->dG + q * M;
    double gR[4], gs = 0.0;
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int x = 0; x < M; ++x) s += w->dT[c * M + x] * G[x];
      gR[c] = s * inv_nm;
    }
    for (int x = 0; x < M; ++x) {
      double s = 0.0;
      for (int c = 0; c < 4; ++c) s += w->dT[c * M + x] * R[c];
      gs += s * dG[x];
    }
    gs *= inv_nm;
    /* s = R[0] itself depends on r: dR_0/dd = ds/dr u, so the G-path term
     * enters through the same derivative as R[0] */
    double gr0 = gR[0] + gs;
    for (int b = 0; b < 3; ++b) {
      double v = gr0 * dR[0 * 3 + b];
      for (int a = 0; a < 3; ++a) v += gR[1 + a] * dR[(1 + a) * 3 + b];
      g_out[q * 3 + b] = v;
    }
  }
  return ORC_OK;
}

static int ctx_setup(ctx_t* C, cells_t* cells, const orc_model* m, const orc_table* table,
                     double rc, double rcs, const int32_t* sel, int64_t n, const double* x,
                     const int32_t* types, const double* box) {
  if (!m || !sel || !x || !types || !box || n < 0) return ORC_ERR_ARG;
  if (!(rc > 0) || !(rcs >= 0) || !(rcs < rc)) return ORC_ERR_ARG;
  if (table && (table->M != m->M || table->ntypes != m->ntypes)) return ORC_ERR_ARG;
  double L[3];
  int e = box_lengths(box, L);
  if (e) return e;
  memset(C, 0, sizeof(*C));
  C->m = m;
  C->tab = table;
  C->rc = rc;
  C->rcs = rcs;
  C->sel = sel;
  C->types = types;
  for (int t = 0; t < m->ntypes; ++t) {
    if (sel[t] < 0) return ORC_ERR_ARG;
    C->Nm += sel[t];
  }
  if (C->Nm <= 0) return ORC_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (types[i] < 0 || types[i] >= m->ntypes) return ORC_ERR_ARG;
  e = cells_build(cells, n, x, L, rc);
  if (e) {
    cells_free(cells);
    return e;
  }
  C->cells = cells;
  return ORC_OK;
}

static int64_t cap_for(const ctx_t* C) {
  int64_t cap = 0;
  for (int t = 0; t < C->m->ntypes; ++t) cap += C->sel[t];
  return 4 * cap + 64; /* room to detect and report sel overflow */
}

/* Neumaier compensated sum in index order */
static double neumaier(const double* v, int64_t n) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = s + v[i];
    if (fabs(s) >= fabs(v[i]))
      c += (s - t) + v[i];
    else
      c += (v[i] - t) + s;
    s = t;
  }
  return s + c;
}

int orc_eval(const orc_model* m, const orc_table* table, double rc, double rcs,
             const int32_t* sel, int64_t n, const double* x, const int32_t* types,
             const double* box, double* energy, double* atom_energy, double* force,
             double* virial, int64_t* diag) {
  ctx_t C;
  cells_t cells;
  int e = ctx_setup(&C, &cells, m, table, rc, rcs, sel, n, x, types, box);
  if (e) return e;
  int64_t cap = cap_for(&C);
  double* Ei = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* g = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * cap * 3);
  nbr_t* nb = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)(n > 0 ? n : 1) * cap);
  int64_t* nn = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int* fl = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
  if (!Ei || !g || !nb || !nn || !fl) {
    e = ORC_ERR_NOMEM;
    goto done;
  }
#pragma omp parallel reduction(| : e)
  {
    work_t w;
    int we = work_init(&w, m, cap);
    if (we) {
      e |= we;
    } else {
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        e |= atom_eval(&C, i, &w, &Ei[i], g + (size_t)i * cap * 3, &nn[i], &fl[i]);
        memcpy(nb + (size_t)i * cap, w.nb, sizeof(nbr_t) * (size_t)nn[i]);
      }
    }
    work_free(&w);
  }
  if (e) goto done;
  {
    int64_t maxnn = 0, npairs = 0, nrange = 0, nsel = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (nn[i] > maxnn) maxnn = nn[i];
      npairs += nn[i];
      if (fl[i] & 1) nsel++;
      if (fl[i] & 2) nrange++;
    }
    if (diag) {
      diag[0] = maxnn;
      diag[1] = npairs;
      diag[2] = nrange;
      diag[3] = nsel;
    }
    *energy = neumaier(Ei, n);
    if (atom_energy) memcpy(atom_energy, Ei, sizeof(double) * (size_t)n);
    /* F_i += g_ij, F_j -= g_ij; virial -sum r_ij (x) g_ij; fixed serial order */
    for (int64_t i = 0; i < 3 * n; ++i) force[i] = 0.0;
    double vir[9] = {0};
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = 0; q < nn[i]; ++q) {
        const double* gi = g + ((size_t)i * cap + q) * 3;
        const nbr_t* b = nb + (size_t)i * cap + q;
        for (int a = 0; a < 3; ++a) {
          force[i * 3 + a] += gi[a];
          force[b->j * 3 + a] -= gi[a];
        }
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) vir[a * 3 + c] -= b->d[a] * gi[c];
      }
    if (virial) memcpy(virial, vir, sizeof(vir));
    if (nsel) e = ORC_ERR_SEL;
    else if (nrange) e = ORC_ERR_TABLE_RANGE;
  }
done:
  free(Ei);
  free(g);
  free(nb);
  free(nn);
  free(fl);
  cells_free(&cells);
  return e;
}

int orc_atom_descriptor(const orc_model* m, const orc_table* table, double rc, double rcs,
                        const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                        const double* box, int64_t i, double* T, double* D) {
  ctx_t C;
  cells_t cells;
  int e = ctx_setup(&C, &cells, m, table, rc, rcs, sel, n, x, types, box);
  if (e) return e;
  if (i < 0 || i >= n) {
    cells_free(&cells);
    return ORC_ERR_ARG;
  }
  work_t w;
  e = work_init(&w, m, cap_for(&C));
  if (!e) {
    double Ei;
    int64_t k;
    int fl = 0;
    e = atom_eval(&C, i, &w, &Ei, NULL, &k, &fl);
    if (!e) {
      if (T) memcpy(T, w.T, sizeof(double) * 4 * (size_t)m->M);
      if (D) memcpy(D, w.D, sizeof(double) * (size_t)m->din);
      if (fl & 1) e = ORC_ERR_SEL;
      else if (fl & 2) e = ORC_ERR_TABLE_RANGE;
    }
  }
  work_free(&w);
  cells_free(&cells);
  return e;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

int orc_eval_subset(const orc_model* m, const orc_table* table, double rc, double rcs,
                    const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                    const double* box, int64_t ne, const int64_t* idx_e, double* e_out,
                    int64_t nf, const int64_t* idx_f, double* f_out) {
  ctx_t C;
  cells_t cells;
  int e = ctx_setup(&C, &cells, m, table, rc, rcs, sel, n, x, types, box);
  if (e) return e;
  int64_t cap = cap_for(&C);
  for (int64_t q = 0; q < ne; ++q)
    if (idx_e[q] < 0 || idx_e[q] >= n) e = ORC_ERR_ARG;
  for (int64_t q = 0; q < nf; ++q)
    if (idx_f[q] < 0 || idx_f[q] >= n) e = ORC_ERR_ARG;
  if (e) {
    cells_free(&cells);
    return e;
  }
  /* energies */
#pragma omp parallel reduction(| : e)
  {
    work_t w;
    int we = work_init(&w, m, cap);
    if (we) {
      e |= we;
    } else {
#pragma omp for schedule(dynamic, 8)
      for (int64_t q = 0; q < ne; ++q) {
        int64_t k;
        int fl = 0;
        e |= atom_eval(&C, idx_e[q], &w, &e_out[q], NULL, &k, &fl);
        if (fl & 1) e |= ORC_ERR_SEL;
        if (fl & 2) e |= ORC_ERR_TABLE_RANGE;
      }
    }
    work_free(&w);
  }
  if (e || nf == 0) {
    cells_free(&cells);
    return e;
  }
  /* centres needed for the forces: each target and its neighbors within rc */
  nbr_t* tmp = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)cap);
  int64_t ncent = 0, ccap = nf * (cap + 1);
  int64_t* cent = (int64_t*)malloc(sizeof(int64_t) * (size_t)ccap);
  if (!tmp || !cent) {
    free(tmp);
    free(cent);
    cells_free(&cells);
    return ORC_ERR_NOMEM;
  }
  for (int64_t q = 0; q < nf; ++q) {
    cent[ncent++] = idx_f[q];
    int64_t k = cells_neighbors(&cells, idx_f[q], rc, tmp, cap);
    if (k > cap) k = cap;
    for (int64_t p = 0; p < k; ++p) cent[ncent++] = tmp[p].j;
  }
  free(tmp);
  qsort(cent, (size_t)ncent, sizeof(int64_t), cmp_i64);
  int64_t u = 0;
  for (int64_t q = 0; q < ncent; ++q)
    if (q == 0 || cent[q] != cent[q - 1]) cent[u++] = cent[q];
  ncent = u;
  double* g = (double*)malloc(sizeof(double) * (size_t)ncent * cap * 3);
  nbr_t* nb = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)ncent * cap);
  int64_t* nn = (int64_t*)calloc((size_t)ncent, sizeof(int64_t));
  if (!g || !nb || !nn) {
    e = ORC_ERR_NOMEM;
  } else {
#pragma omp parallel reduction(| : e)
    {
      work_t w;
      int we = work_init(&w, m, cap);
      if (we) {
        e |= we;
      } else {
#pragma omp for schedule(dynamic, 8)
        for (int64_t q = 0; q < ncent; ++q) {
          double Ei;
          int fl = 0;
          e |= atom_eval(&C, cent[q], &w, &Ei, g + (size_t)q * cap * 3, &nn[q], &fl);
          memcpy(nb + (size_t)q * cap, w.nb, sizeof(nbr_t) * (size_t)nn[q]);
          if (fl & 1) e |= ORC_ERR_SEL;
          if (fl & 2) e |= ORC_ERR_TABLE_RANGE;
        }
      }
      work_free(&w);
    }
  }
  if (!e) {
    for (int64_t q = 0; q < nf; ++q) {
      int64_t k = idx_f[q];
      double F[3] = {0, 0, 0};
      for (int64_t c = 0; c < ncent; ++c) {
        int64_t i = cent[c];
        for (int64_t p = 0; p < nn[c]; ++p) {
          const double* gi = g + ((size_t)c * cap + p) * 3;
          if (i == k)
            for (int a = 0; a < 3; ++a) F[a] += gi[a];
          if (nb[(size_t)c * cap + p].j == k)
            for (int a = 0; a < 3; ++a) F[a] -= gi[a];
        }
      }
      for (int a = 0; a < 3; ++a) f_out[q * 3 + a] = F[a];
    }
  }
  free(g);
  free(nb);
  free(nn);
  free(cent);
  cells_free(&cells);
  return e;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: velocity-Verlet NVE                                                */
/* ------------------------------------------------------------------------ */
#define ORC_ACC 9.648533212e-3 /* (eV/A/amu) -> A/fs^2 */
#define ORC_KB 8.617333262e-5  /* eV/K */
#define ORC_EVA3_BAR 1.602176634e6

static void thermo_row(int64_t n, const double* v, const int32_t* types, const double* mass,
                       double pe, const double* vir, double vol, double* row) {
  double ke = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double m = mass[types[i]];
    ke += 0.5 * m * (v[i * 3] * v[i * 3] + v[i * 3 + 1] * v[i * 3 + 1] + v[i * 3 + 2] * v[i * 3 + 2]);
  }
  ke /= ORC_ACC;
  int64_t dof = 3 * n - 3;
  row[0] = ke;
  row[1] = pe;
  row[2] = dof > 0 ? 2.0 * ke / (dof * ORC_KB) : 0.0;
  row[3] = (2.0 * ke + vir[0] + vir[4] + vir[8]) / (3.0 * vol) * ORC_EVA3_BAR;
}

int orc_md(const orc_model* m, const orc_table* table, double rc, double rcs,
           const int32_t* sel, int64_t n, double* x, double* v, double* f, int f_valid,
           const int32_t* types, const double* mass_of_type, const double* box,
           double dt, int nsteps, double* thermo) {
  if (!m || !x || !v || !f || !mass_of_type || nsteps < 0) return ORC_ERR_ARG;
  double vol = box[0] * box[4] * box[8];
  double pe = 0.0, vir[9] = {0};
  int e = 0;
  if (!f_valid) e = orc_eval(m, table, rc, rcs, sel, n, x, types, box, &pe, NULL, f, vir, NULL);
  if (e) return e;
  if (thermo) thermo_row(n, v, types, mass_of_type, pe, vir, vol, thermo);
  for (int s = 0; s < nsteps; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      double a = 0.5 * dt * ORC_ACC / mass_of_type[types[i]];
      for (int c = 0; c < 3; ++c) {
        v[i * 3 + c] += a * f[i * 3 + c];
        x[i * 3 + c] += dt * v[i * 3 + c];
      }
    }
    e = orc_eval(m, table, rc, rcs, sel, n, x, types, box, &pe, NULL, f, vir, NULL);
    if (e) return e;
    for (int64_t i = 0; i < n; ++i) {
      double a = 0.5 * dt * ORC_ACC / mass_of_type[types[i]];
      for (int c = 0; c < 3; ++c) v[i * 3 + c] += a * f[i * 3 + c];
    }
    if (thermo) thermo_row(n, v, types, mass_of_type, pe, vir, vol, thermo + (size_t)(s + 1) * 4);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Parameter gradients: dE/d(fitting weights, biases) and dE/d(table        */
/* coefficients) of the same energy (Sec. 2.1 network, Sec. 3.2 table)      */
/* ------------------------------------------------------------------------ */
/* per centre type: layer k as a [(win_k + 1)][wout_k] block (W_k rows, then
 * b_k), then w_out and b_out as a [(w_last + 1)] block */
int64_t orc_fit_param_count(const orc_model* m) {
  if (!m) return -ORC_ERR_ARG;
  int64_t c = 0;
  int win = m->din;
  for (int k = 0; k < m->n_fit; ++k) {
    c += (int64_t)(win + 1) * m->fit_w[k];
    win = m->fit_w[k];
  }
  return c + win + 1;
}

int orc_model_fit_params(orc_model* m, int ti, double* get, const double* set) {
  if (!m || ti < 0 || ti >= m->ntypes) return ORC_ERR_ARG;
  int64_t o = 0;
  int win = m->din;
  for (int k = 0; k < m->n_fit; ++k) {
    const int wo = m->fit_w[k];
    double* W = (double*)m->fit_W[ti][k];
    double* b = (double*)m->fit_b[ti][k];
    const size_t nw = (size_t)win * wo;
    if (get) {
      memcpy(get + o, W, sizeof(double) * nw);
      memcpy(get + o + nw, b, sizeof(double) * wo);
    }
    if (set) {
      memcpy(W, set + o, sizeof(double) * nw);
      memcpy(b, set + o + nw, sizeof(double) * wo);
    }
    o += (int64_t)nw + wo;
    win = wo;
  }
  double* wout = (double*)m->fit_wout[ti];
  if (get) {
    memcpy(get + o, wout, sizeof(double) * win);
    get[o + win] = m->fit_bout[ti];
  }
  if (set) {
    memcpy(wout, set + o, sizeof(double) * win);
    m->fit_bout[ti] = set[o + win];
  }
  return ORC_OK;
}

int orc_table_set_coeffs(orc_table* t, int ti, int tj, const double* in) {
  if (!t || !in || ti < 0 || tj < 0 || ti >= t->ntypes || tj >= t->ntypes) return ORC_ERR_ARG;
  size_t sz = (size_t)t->n * 6 * t->M;
  memcpy(t->a + (size_t)(ti * t->ntypes + tj) * sz, in, sizeof(double) * sz);
  return ORC_OK;
}

/* The fitting net of type ti on D: E, dD = dE/dD and, added into g (the
 * type's block of the gradient), dE/d(parameters).  Chain rule through
 * z_k = [shortcut] z_{k-1} + act(z_{k-1} W_k + b_k), E = z_last . w + b:
 * with gz_k = dE/dz_k and gp_k = gz_k act'(a_k),
 *   dE/dW_k[r][c] = in_k[r] gp_k[c],  dE/db_k = gp_k,
 *   gz_{k-1} = gp_k W_k^T + [shortcut] gz_k,  dE/dw = z_last, dE/db = 1. */
static int fit_grad(const orc_model* m, int ti, const double* D, double* E, double* dD,
                    double* g) {
  const int nf = m->n_fit;
  int wid[MAXL + 1];
  wid[0] = m->din;
  for (int k = 0; k < nf; ++k) wid[k + 1] = m->fit_w[k];
  size_t zoff[MAXL + 1], goff[MAXL + 1];
  zoff[0] = 0;
  goff[0] = 0;
  for (int k = 0; k < nf; ++k) {
    zoff[k + 1] = zoff[k] + (size_t)wid[k + 1];
    goff[k + 1] = goff[k] + (size_t)(wid[k] + 1) * wid[k + 1];
  }
  int wmax = m->din;
  for (int k = 1; k <= nf; ++k) wmax = wid[k] > wmax ? wid[k] : wmax;
  double* z = (double*)malloc(sizeof(double) * (2 * zoff[nf] + 3 * (size_t)wmax));
  if (!z) return ORC_ERR_NOMEM;
  double* dact = z + zoff[nf];
  double* gz = dact + zoff[nf];
  double* gn = gz + wmax;
  double* gp = gn + wmax;
  for (int k = 0; k < nf; ++k) {
    const double* in = k ? z + zoff[k - 1] : D;
    const int wi = wid[k], wo = wid[k + 1];
    const int shortcut = (k > 0 && wo == wi);
    for (int c = 0; c < wo; ++c) {
      double a = m->fit_b[ti][k][c];
      for (int r = 0; r < wi; ++r) a += in[r] * m->fit_W[ti][k][(size_t)r * wo + c];
      double da;
      const double t = orc_act(a, &da);
      dact[zoff[k] + c] = da;
      z[zoff[k] + c] = (shortcut ? in[c] : 0.0) + t;
    }
  }
  const double* zl = z + zoff[nf - 1];
  const int wl = wid[nf];
  double e = m->fit_bout[ti];
  for (int c = 0; c < wl; ++c) e += zl[c] * m->fit_wout[ti][c];
  *E = e;
  double* gout = g + goff[nf];
  for (int c = 0; c < wl; ++c) {
    gout[c] += zl[c];
    gz[c] = m->fit_wout[ti][c];
  }
  gout[wl] += 1.0;
  for (int k = nf - 1; k >= 0; --k) {
    const double* in = k ? z + zoff[k - 1] : D;
    const int wi = wid[k], wo = wid[k + 1];
    const int shortcut = (k > 0 && wo == wi);
    double* gW = g + goff[k];
    double* gb = gW + (size_t)wi * wo;
    for (int c = 0; c < wo; ++c) {
      gp[c] = gz[c] * dact[zoff[k] + c];
      gb[c] += gp[c];
    }
    for (int r = 0; r < wi; ++r) {
      double s = shortcut ? gz[r] : 0.0;
      for (int c = 0; c < wo; ++c) {
        gW[(size_t)r * wo + c] += in[r] * gp[c];
        s += m->fit_W[ti][k][(size_t)r * wo + c] * gp[c];
      }
      gn[r] = s;
    }
    double* sw = gz;
    gz = gn;
    gn = sw;
  }
  memcpy(dD, gz, sizeof(double) * m->din);
  free(z);
  return ORC_OK;
}

/* per (centre type, neighbor type) embedding net: layer k as a
 * [(win_k + 1)][wout_k] block (W_k rows, then b_k), win_0 = 1 */
int64_t orc_emb_param_count(const orc_model* m) {
  if (!m) return -ORC_ERR_ARG;
  int64_t c = 0;
  int win = 1;
  for (int k = 0; k < m->n_emb; ++k) {
    c += (int64_t)(win + 1) * m->emb_w[k];
    win = m->emb_w[k];
  }
  return c;
}

int orc_model_emb_params(orc_model* m, int ti, int tj, double* get, const double* set) {
  if (!m || ti < 0 || tj < 0 || ti >= m->ntypes || tj >= m->ntypes) return ORC_ERR_ARG;
  const int p = ti * m->ntypes + tj;
  int64_t o = 0;
  int win = 1;
  for (int k = 0; k < m->n_emb; ++k) {
    const int wo = m->emb_w[k];
    double* W = (double*)m->emb_W[p][k];
    double* b = (double*)m->emb_b[p][k];
    const size_t nw = (size_t)win * wo;
    if (get) {
      memcpy(get + o, W, sizeof(double) * nw);
      memcpy(get + o + nw, b, sizeof(double) * wo);
    }
    if (set) {
      memcpy(W, set + o, sizeof(double) * nw);
      memcpy(b, set + o + nw, sizeof(double) * wo);
    }
    o += (int64_t)nw + wo;
    win = wo;
  }
  return ORC_OK;
}

/* dE/d(embedding-net parameters of pair type p) added into g, given
 * dE/dG at s.  Reverse mode through Eq. 4-5: with out_L = (in,in) + t_L,
 * t_L = tanh(in W_L + b_L) and dz = dE/dout_L (1 - t_L^2):
 *   dE/dW_L[k][c] = in[k] dz[c],  dE/db_L = dz,
 *   dE/din[k] = sum_c W_L[k][c] dz[c] + sum_{c : c mod win = k} dE/dout_L[c]. */
static int emb_grad(const orc_model* m, int p, double s, const double* dEdG, double* g) {
  const int nl = m->n_emb;
  size_t tot = 0;
  for (int k = 0; k < nl; ++k) tot += (size_t)m->emb_w[k];
  double* buf = (double*)malloc(sizeof(double) * (2 * tot + 3 * (size_t)m->M));
  if (!buf) return ORC_ERR_NOMEM;
  double* t = buf;         /* tanh values, layer by layer */
  double* out = buf + tot; /* layer outputs */
  double* d = out + tot;
  double* dn = d + m->M;
  double* dz = dn + m->M;
  size_t off[MAXL + 1];
  off[0] = 0;
  for (int k = 0; k < nl; ++k) off[k + 1] = off[k] + (size_t)m->emb_w[k];
  for (int c = 0; c < m->emb_w[0]; ++c) {
    t[c] = tanh(s * m->emb_W[p][0][c] + m->emb_b[p][0][c]);
    out[c] = t[c];
  }
  for (int L = 1; L < nl; ++L) {
    const int win = m->emb_w[L - 1], wo = m->emb_w[L];
    const double* in = out + off[L - 1];
    for (int c = 0; c < wo; ++c) {
      double z = m->emb_b[p][L][c];
      for (int k = 0; k < win; ++k) z += in[k] * m->emb_W[p][L][(size_t)k * wo + c];
      t[off[L] + c] = tanh(z);
      out[off[L] + c] = in[c % win] + t[off[L] + c];
    }
  }
  size_t goff[MAXL + 1];
  goff[0] = 0;
  for (int k = 0, win = 1; k < nl; ++k) {
    goff[k + 1] = goff[k] + (size_t)(win + 1) * m->emb_w[k];
    win = m->emb_w[k];
  }
  memcpy(d, dEdG, sizeof(double) * m->M);
  for (int L = nl - 1; L >= 1; --L) {
    const int win = m->emb_w[L - 1], wo = m->emb_w[L];
    const double* in = out + off[L - 1];
    double* gW = g + goff[L];
    double* gb = gW + (size_t)win * wo;
    for (int c = 0; c < wo; ++c) {
      const double tt = t[off[L] + c];
      dz[c] = d[c] * (1.0 - tt * tt);
      gb[c] += dz[c];
    }
    for (int k = 0; k < win; ++k) {
      double v = 0.0;
      for (int c = 0; c < wo; ++c) {
        gW[(size_t)k * wo + c] += in[k] * dz[c];
        v += m->emb_W[p][L][(size_t)k * wo + c] * dz[c];
      }
      for (int c = k; c < wo; c += win) v += d[c];
      dn[k] = v;
    }
    memcpy(d, dn, sizeof(double) * win);
  }
  const int w0 = m->emb_w[0];
  for (int c = 0; c < w0; ++c) {
    const double dz0 = d[c] * (1.0 - t[c] * t[c]);
    g[c] += s * dz0;       /* W_0 [1][w0] */
    g[w0 + c] += dz0;      /* b_0 */
  }
  free(buf);
  return ORC_OK;
}

/* E and the parameter gradients of the whole system.  grad_fit: the blocks
 * of every centre type in type order (orc_fit_param_count each).
 * grad_table (tabulated model only, may be NULL): [ntypes*ntypes][n][6][M]
 * with respect to the coefficients c_q = a_q h^q of the normalised local
 * variable v = (s - k h)/h, the form the CUDA library stores.  Since
 *   T_i[c][x] = (1/N_m) sum_j R_jc sum_q c_q[x] v_j^q,
 * dE/dc[k][q][x] = (1/N_m) sum_i sum_{j in interval k} (sum_c dE/dT_i[c][x] R_jc) v_j^q.
 * Serial over atoms (a fixed summation order). */
int orc_param_grad(const orc_model* m, const orc_table* table, double rc, double rcs,
                   const int32_t* sel, int64_t n, const double* x, const int32_t* types,
                   const double* box, double* energy, double* grad_fit, double* grad_table) {
  if (!grad_fit || !energy) return ORC_ERR_ARG;
  ctx_t C;
  cells_t cells;
  int e = ctx_setup(&C, &cells, m, table, rc, rcs, sel, n, x, types, box);
  if (e) return e;
  const int64_t per = orc_fit_param_count(m);
  const int M = m->M, mlt = m->m_lt;
  memset(grad_fit, 0, sizeof(double) * (size_t)per * m->ntypes);
  const int64_t per_emb = orc_emb_param_count(m);
  if (grad_table)
    memset(grad_table, 0,
           sizeof(double) * (size_t)m->ntypes * m->ntypes *
               (table ? (size_t)table->n * 6 * M : (size_t)per_emb));
  const double inv_nm = 1.0 / (double)C.Nm;
  work_t w;
  double* Ei = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* dEdg = (double*)malloc(sizeof(double) * (size_t)M);
  e = work_init(&w, m, cap_for(&C));
  if (!Ei || !dEdg) e = e ? e : ORC_ERR_NOMEM;
  int flags = 0;
  for (int64_t i = 0; i < n && !e; ++i) {
    const int ti = types[i];
    int64_t k = cells_neighbors(C.cells, i, rc, w.nb, w.cap);
    if (k > w.cap) {
      e = ORC_ERR_SEL;
      break;
    }
    int cnt_t[MAXT] = {0};
    for (int64_t q = 0; q < k; ++q) cnt_t[types[w.nb[q].j]]++;
    for (int t = 0; t < m->ntypes; ++t)
      if (cnt_t[t] > sel[t]) flags |= 1;
    /* T (Eq. 1 rows, table or net, 1/N_m) and D (Eq. 2), as orc_eval */
    for (int c = 0; c < 4 * M; ++c) w.T[c] = 0.0;
    for (int64_t q = 0; q < k; ++q) {
      const int tj = types[w.nb[q].j];
      double* R = w.R + q * 4;
      const double s = orc_env_row(w.nb[q].d, rc, rcs, R, w.dR + q * 12);
      double* G = w.G + q * M;
      if (table) {
        if (orc_table_eval(table, ti, tj, s, G, w.dG + q * M)) flags |= 2;
      } else {
        orc_embed(m, ti, tj, s, G, w.dG + q * M, NULL);
      }
      for (int c = 0; c < 4; ++c)
        for (int a = 0; a < M; ++a) w.T[c * M + a] += R[c] * G[a] * inv_nm;
    }
    for (int b = 0; b < M; ++b)
      for (int a = 0; a < mlt; ++a) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) s += w.T[c * M + b] * w.T[c * M + a];
        w.D[b * mlt + a] = s;
      }
    e = fit_grad(m, ti, w.D, &Ei[i], w.dD, grad_fit + (size_t)ti * per);
    if (e || !grad_table) continue;
    /* dE/dT from dE/dD (both factors of Eq. 2) */
    for (int c = 0; c < 4; ++c)
      for (int a = 0; a < M; ++a) {
        double s = 0.0;
        for (int b = 0; b < mlt; ++b) s += w.dD[a * mlt + b] * w.T[c * M + b];
        if (a < mlt)
          for (int b = 0; b < M; ++b) s += w.dD[b * mlt + a] * w.T[c * M + b];
        w.dT[c * M + a] = s;
      }
    for (int64_t q = 0; q < k && !e; ++q) {
      const int tj = types[w.nb[q].j];
      const double* R = w.R + q * 4;
      const double s = R[0];
      for (int a = 0; a < M; ++a) {
        double g = 0.0;
        for (int c = 0; c < 4; ++c) g += w.dT[c * M + a] * R[c];
        dEdg[a] = g * inv_nm;
      }
      if (!table) {
        /* the original embedding net: its weights and biases */
        e = emb_grad(m, ti * m->ntypes + tj, s, dEdg,
                     grad_table + (size_t)(ti * m->ntypes + tj) * per_emb);
        continue;
      }
      /* the interval and local variable of orc_table_eval, the latter
       * normalised by the interval's width */
      int kk;
      const double v = tab_locate(table, s, &kk) / tab_width(table, kk);
      double* out = grad_table + ((size_t)(ti * m->ntypes + tj) * table->n + kk) * 6 * M;
      double vp = 1.0;
      for (int p = 0; p < 6; ++p) {
        for (int a = 0; a < M; ++a) out[p * M + a] += dEdg[a] * vp;
        vp *= v;
      }
    }
  }
  if (!e) {
    *energy = neumaier(Ei, n);
    if (flags & 1) e = ORC_ERR_SEL;
    else if (flags & 2) e = ORC_ERR_TABLE_RANGE;
  }
  work_free(&w);
  free(Ei);
  free(dEdg);
  cells_free(&cells);
  return e;
}
