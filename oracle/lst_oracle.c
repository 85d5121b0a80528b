/*
 * CPU oracle for the Line Segment Tracking hot path -- TEST INFRASTRUCTURE ONLY
 * (used by tests/, the smoke check and the benchmark's CPU-baseline leg; never by the
 * CUDA library, which shares no code with this file).
 *
 * Build: cc -O2 -std=c99 -ffp-contract=off -fno-fast-math -fPIC -shared -lm -lpthread.
 * Arithmetic: IEEE binary32, every expression evaluated left to right as written, only
 * + - * / sqrtf fabsf and comparisons in the cut code (no FMA contraction, no flush to
 * zero).  Angle-dependent module constants are computed once in double and rounded.
 *
 * What the paper fixes (arXiv:2407.18231, Sec. 1):
 *   - every outer-tracker layer is two closely spaced sensors; a Mini Doublet (MD) pairs
 *     a hit on each sensor of one module, with a window tuned for pT >= 0.8 GeV;
 *   - precomputed module connection maps decide which MDs may be linked into a Line
 *     Segment (LS); two LSs sharing an MD form a T3; two T3s sharing an MD form a T5;
 *   - T3s and T5s are combined with inner-tracker tracks (pLS) into pT3s and pT5s;
 *   - only a subset is propagated: pT5s, pT3s, T5s and unlinked pLSs (track candidates);
 *   - T5s carry no beam-line requirement (displaced tracks, Sec. 2-3).
 * Everything numeric below (cut forms, tolerances, the duplicate rule) is this
 * project's reading: the paper defers the selections to its references.  Each reading
 * is stated at the function that applies it.
 *
 * Object order ("canonical"): hits of a sensor by (pseudo-angle, input index); MDs by
 * (module, lower hit, upper hit) in that order; LS by (inner MD, outer MD); T3 by (MD a, b,
 * c); T5 by (a..e); pT3/pT5 by (pLS, T3/T5 index); TCs by type pT5, pT3, T5, pLS then index.
 */
#include "lst_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- constants (units cm, GeV, T) ---------------- */
#define KB_D (0.0029979245800 * 3.8) /* pT = KB * R */
#define PTMIN_D 0.8                  /* lower pT threshold (Sec. 1) */
#define RMIN_D (PTMIN_D / KB_D)      /* minimum curvature radius, 70.2 cm */
#define NSURF 16

static const float C_KB = (float)KB_D;
static const float C_Z0MAX = 15.0f;                                  /* 3 sigma of the 5 cm luminous region */
static const float C_E0 = 0.03f;                                     /* r-phi tolerance of a hit pair */
static const float C_KARC = (float)(2.0 / (24.0 * RMIN_D * RMIN_D)); /* arc-vs-chord bound, margin 2 */
static const float C_K3 = (float)(2.0 * RMIN_D * 0.95);              /* 2 Rmin (1 - 5 %) */
static const float C_KMAX = (float)(1.0 / (RMIN_D * 0.95));          /* largest accepted curvature */
static const float C_KAPPA = 0.05f;                                  /* relative curvature consistency */
static const float C_KAPPA0 = 1.0e-4f;                               /* absolute curvature slack, 1/cm */
static const float C_KPT5 = 0.15f;                                   /* pT5: T5 vs pLS curvature */
static const float C_W0 = 0.02f;                                     /* pLS r-phi window floor */
static const float C_PI = 3.14159265f;
static const float C_HINV = (float)(1.0 / (2.0 * RMIN_D));           /* sin(tangent, chord) per cm of chord */
static const float C_EDIR = 0.013f;                                  /* 3 sqrt(2) x 30 um across an MD */

/* ---------------- small growable arrays ---------------- */
typedef struct { uint32_t *p; size_t n, cap; } vu32;
typedef struct { float *p; size_t n, cap; } vf32;

static int vu32_push(vu32 *v, uint32_t x) {
  if (v->n == v->cap) {
    size_t c = v->cap ? 2 * v->cap : 256;
    uint32_t *q = (uint32_t *)realloc(v->p, c * sizeof(uint32_t));
    if (!q) return -1;
    v->p = q; v->cap = c;
  }
  v->p[v->n++] = x;
  return 0;
}
static int vf32_push(vf32 *v, float x) {
  if (v->n == v->cap) {
    size_t c = v->cap ? 2 * v->cap : 256;
    float *q = (float *)realloc(v->p, c * sizeof(float));
    if (!q) return -1;
    v->p = q; v->cap = c;
  }
  v->p[v->n++] = x;
  return 0;
}

/* ---------------- geometry ---------------- */
struct ora_geom {
  uint32_t n;
  ora_module *m;
  int *surface;                 /* 0..5 barrel layers, 6..10 disks z<0, 11..15 disks z>0 */
  float *T, *zeta, *rho, *delta;/* per-module cut constants */
  float *rnext;                 /* barrel: lower radius of the next barrel layer (1e30: none) */
  float zb_half;                /* barrel half length */
  /* per surface: rows (z bin or ring) of modules indexed by iphi */
  uint32_t n_rows[NSURF];
  uint32_t *row_nphi[NSURF];
  uint32_t **row_mod[NSURF];
  uint32_t *surf_list[NSURF];   /* module ids of each surface, ascending */
  uint32_t surf_count[NSURF];
  uint32_t *row_off, *cols;     /* connection map (CSR) */
  float *t5_mlp;                /* learned T5 selection (ORA_T5_NPARAM weights), NULL = cuts */
};

static int module_surface(const ora_module *m) {
  if (m->subdet == 0) return (m->layer >= 1 && m->layer <= 6) ? m->layer - 1 : -1;
  if (m->subdet == 1 && m->layer >= 1 && m->layer <= 5) {
    if (m->side < 0) return 6 + m->layer - 1;
    if (m->side > 0) return 11 + m->layer - 1;
  }
  return -1;
}

/* Surfaces a track can cross next when it moves outward from surface s: the next barrel
 * layer, the first disk on either side, or the next disk on the same side. */
static int next_surfaces(int s, int out[3]) {
  int k = 0;
  if (s < 6) {
    if (s < 5) out[k++] = s + 1;
    out[k++] = 6;
    out[k++] = 11;
  } else if (s < 11) {
    if (s < 10) out[k++] = s + 1;
  } else {
    if (s < 15) out[k++] = s + 1;
  }
  return k;
}

/* Per-module constants (reading of the pT >= 0.8 GeV window, Sec. 1):
 *   T     = tan(asin(r_max / (2 Rmin))): largest angle between a prompt pT >= 0.8 GeV
 *           track's chord ending at radius r_max and the radial direction at its start
 *           (r_max: the module's largest radius, the upper sensor of a tilted module
 *           included);
 *   zeta  = z tolerance of one hit (PS 3 x 0.5 mm, 2S half a 2.5 cm strip + 0.5 mm);
 *   rho   = radial tolerance of one hit (endcap PS 3 x 0.5 mm, endcap 2S half a 5 cm
 *           strip + 0.5 mm);
 *   delta = transverse point tolerance (3 x 30 um rounded up, plus rho).
 * A tilted barrel PS module (Fig. 1) measures its coarse coordinate along its surface,
 * direction (-sin t, cos t) in r-z: 3 x 0.5 mm projects to zeta = 0.15 |cos t| and
 * rho = 0.15 |sin t|; its lower sensor spans r in surf +- (half its z length) |tan t|. */
static void module_consts(const ora_module *m, float *T, float *zeta, float *rho, float *delta) {
  double rmax;
  if (m->subdet == 0) {
    double t = (double)m->tilt;
    rmax = (double)m->surf + 0.5 * ((double)m->emax - (double)m->emin) * fabs(tan(t)) + (double)m->gap * cos(t);
  } else {
    rmax = (double)m->emax;
  }
  double s = rmax / (2.0 * RMIN_D);
  *T = (float)(s < 1.0 ? s / sqrt(1.0 - s * s) : 1.0e30);
  if (m->subdet == 0) {
    if (m->tilt != 0.0f) {
      *zeta = (float)(0.15 * fabs(cos((double)m->tilt)));
      *rho = (float)(0.15 * fabs(sin((double)m->tilt)));
    } else {
      *zeta = m->stype == 0 ? 0.15f : 1.30f;
      *rho = 0.0f;
    }
  } else {
    *zeta = 0.0f;
    *rho = m->stype == 0 ? 0.15f : 2.55f;
  }
  *delta = 0.01f + *rho;
}

/* Anchor coordinate box of a module (lower sensor, with margins for resolution). */
static void anchor_box(const ora_module *m, double *r0, double *r1, double *z0, double *z1) {
  if (m->subdet == 0 && m->tilt != 0.0f) {
    double h = 0.5 * ((double)m->emax - (double)m->emin) * fabs(tan((double)m->tilt));
    *r0 = m->surf - h - 0.5; *r1 = m->surf + h + 0.5;
    *z0 = m->emin - 0.5; *z1 = m->emax + 0.5;
  } else if (m->subdet == 0) {
    *r0 = m->surf - 0.01; *r1 = m->surf + 0.01;
    *z0 = m->emin - 0.5; *z1 = m->emax + 0.5;
  } else {
    *z0 = m->surf - 0.01; *z1 = m->surf + 0.01;
    *r0 = m->emin - 0.5; *r1 = m->emax + 0.5;
  }
}

static double wedge_centre(const ora_module *m, double *half) {
  double a0 = atan2(m->e0y, m->e0x);
  double a1 = atan2(m->e1y, m->e1x);
  double w = a1 - a0;
  while (w <= 0) w += 2 * M_PI;
  *half = 0.5 * w;
  return a0 + 0.5 * w;
}

/* Connection map (Sec. 1: MDs are linked only between modules that a map, built ahead
 * of time from the geometry, marks as reachable by real tracks).  Reading: B is connected to A
 * when B lies on a surface next to A's and the LS selection below can be met by some
 * pair of anchors inside the two modules.  The test is conservative (bounds the LS cut
 * over the anchor boxes), so the map only prunes pairs that could never pass. */
static int map_ok(const ora_geom *g, uint32_t A, uint32_t B) {
  const ora_module *ma = &g->m[A], *mb = &g->m[B];
  double rA0, rA1, zA0, zA1, rB0, rB1, zB0, zB1;
  anchor_box(ma, &rA0, &rA1, &zA0, &zA1);
  anchor_box(mb, &rB0, &rB1, &zB0, &zB1);
  /* phi: |tan(dphi)| <= T_B + e_max / (r_a - rho_sum) follows from the bending cut */
  double rs = (double)g->rho[A] + (double)g->rho[B];
  double emax = 0.03 + rs * 1.05;
  double dphi = atan((double)g->T[B] + emax / (rA0 - rs)) + 3.0e-3;
  double hA, hB;
  double cA = wedge_centre(ma, &hA), cB = wedge_centre(mb, &hB);
  double dc = remainder(cA - cB, 2 * M_PI);
  if (fabs(dc) > hA + hB + dphi) return 0;
  /* r-z: min |za rb - ra zb| over the box against max of the tolerance over the box */
  double flo = 1e300, fhi = -1e300;
  double zas[2] = {zA0, zA1}, ras[2] = {rA0, rA1}, zbs[2] = {zB0, zB1}, rbs[2] = {rB0, rB1};
  for (int i = 0; i < 16; i++) {
    double f = zas[i & 1] * rbs[(i >> 3) & 1] - ras[(i >> 1) & 1] * zbs[(i >> 2) & 1];
    if (f < flo) flo = f;
    if (f > fhi) fhi = f;
  }
  double lhs = (flo <= 0 && fhi >= 0) ? 0.0 : fmin(fabs(flo), fabs(fhi));
  double drmax = fmax(fabs(rB1 - rA0), fabs(rB0 - rA1));
  double zbmax = fmax(fabs(zB0), fabs(zB1)), zamax = fmax(fabs(zA0), fabs(zA1));
  double dzmax = fmax(fabs(zB1 - zA0), fabs(zB0 - zA1));
  double rhs = 15.0 * drmax + g->zeta[A] * rB1 + g->zeta[B] * rA1 + g->rho[A] * zbmax +
               g->rho[B] * zamax + (double)C_KARC * dzmax * rA1 * rB1 * (rA1 + rB1);
  return lhs <= rhs * 1.01 + 0.01;
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : x > y;
}

void ora_geom_destroy(ora_geom *g) {
  if (!g) return;
  for (int s = 0; s < NSURF; s++) {
    if (g->row_mod[s]) {
      for (uint32_t r = 0; r < g->n_rows[s]; r++) free(g->row_mod[s][r]);
      free(g->row_mod[s]);
    }
    free(g->row_nphi[s]);
    free(g->surf_list[s]);
  }
  free(g->m); free(g->surface); free(g->T); free(g->zeta); free(g->rho); free(g->delta); free(g->rnext);
  free(g->row_off); free(g->cols); free(g->t5_mlp);
  free(g);
}

ora_geom *ora_geom_create(const ora_module *mods, uint32_t n) {
  if (!mods || n == 0) return NULL;
  ora_geom *g = (ora_geom *)calloc(1, sizeof(ora_geom));
  if (!g) return NULL;
  g->n = n;
  g->m = (ora_module *)malloc(n * sizeof(ora_module));
  g->surface = (int *)malloc(n * sizeof(int));
  g->T = (float *)malloc(n * sizeof(float));
  g->zeta = (float *)malloc(n * sizeof(float));
  g->rho = (float *)malloc(n * sizeof(float));
  g->delta = (float *)malloc(n * sizeof(float));
  g->rnext = (float *)malloc(n * sizeof(float));
  if (!g->m || !g->surface || !g->T || !g->zeta || !g->rho || !g->delta || !g->rnext) goto fail;
  memcpy(g->m, mods, n * sizeof(ora_module));
  for (uint32_t i = 0; i < n; i++) {
    const ora_module *m = &g->m[i];
    int s = module_surface(m);
    if (s < 0 || m->nphi == 0 || m->iphi >= m->nphi) goto fail;
    if (!isfinite(m->surf) || !isfinite(m->gap) || !isfinite(m->emin) || !isfinite(m->emax)) goto fail;
    if (!(fabsf(m->tilt) < 1.5f) || (m->subdet != 0 && m->tilt != 0.0f)) goto fail;
    g->surface[i] = s;
    module_consts(m, &g->T[i], &g->zeta[i], &g->rho[i], &g->delta[i]);
    if (m->ieta + 1u > g->n_rows[s]) g->n_rows[s] = m->ieta + 1u;
    g->surf_count[s]++;
  }
  {
    float rlay[6];
    int have[6] = {0, 0, 0, 0, 0, 0};
    g->zb_half = 0.0f;
    for (uint32_t i = 0; i < n; i++) {
      const ora_module *m = &g->m[i];
      if (m->subdet != 0) continue;
      rlay[m->layer - 1] = m->surf;
      have[m->layer - 1] = 1;
      if (fabsf(m->emin) > g->zb_half) g->zb_half = fabsf(m->emin);
      if (fabsf(m->emax) > g->zb_half) g->zb_half = fabsf(m->emax);
    }
    for (uint32_t i = 0; i < n; i++) {
      const ora_module *m = &g->m[i];
      g->rnext[i] = 1.0e30f;
      if (m->subdet == 0 && m->layer < 6 && have[m->layer]) g->rnext[i] = rlay[m->layer];
    }
  }
  for (int s = 0; s < NSURF; s++) {
    if (!g->n_rows[s]) continue;
    g->row_nphi[s] = (uint32_t *)calloc(g->n_rows[s], sizeof(uint32_t));
    g->row_mod[s] = (uint32_t **)calloc(g->n_rows[s], sizeof(uint32_t *));
    g->surf_list[s] = (uint32_t *)malloc(g->surf_count[s] * sizeof(uint32_t));
    if (!g->row_nphi[s] || !g->row_mod[s] || !g->surf_list[s]) goto fail;
    g->surf_count[s] = 0;
  }
  for (uint32_t i = 0; i < n; i++) {
    const ora_module *m = &g->m[i];
    int s = g->surface[i];
    g->surf_list[s][g->surf_count[s]++] = i;
    uint32_t **row = &g->row_mod[s][m->ieta];
    if (!*row) {
      g->row_nphi[s][m->ieta] = m->nphi;
      *row = (uint32_t *)malloc(m->nphi * sizeof(uint32_t));
      if (!*row) goto fail;
      for (uint32_t k = 0; k < m->nphi; k++) (*row)[k] = UINT32_MAX;
    }
    if (g->row_nphi[s][m->ieta] != m->nphi || (*row)[m->iphi] != UINT32_MAX) goto fail;
    (*row)[m->iphi] = i;
  }
  /* connection map */
  {
    vu32 cols = {0};
    g->row_off = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    if (!g->row_off) goto fail;
    for (uint32_t A = 0; A < n; A++) {
      g->row_off[A] = (uint32_t)cols.n;
      int nxt[3];
      int k = next_surfaces(g->surface[A], nxt);
      for (int t = 0; t < k; t++) {
        int s = nxt[t];
        for (uint32_t q = 0; q < g->surf_count[s]; q++) {
          uint32_t B = g->surf_list[s][q];
          if (map_ok(g, A, B) && vu32_push(&cols, B)) { free(cols.p); goto fail; }
        }
      }
      qsort(cols.p + g->row_off[A], cols.n - g->row_off[A], sizeof(uint32_t), cmp_u32);
    }
    g->row_off[n] = (uint32_t)cols.n;
    g->cols = cols.p;
  }
  return g;
fail:
  ora_geom_destroy(g);
  return NULL;
}

uint32_t ora_geom_map(const ora_geom *g, const uint32_t **row_off, const uint32_t **cols) {
  *row_off = g->row_off;
  *cols = g->cols;
  return g->row_off[g->n];
}

/* ---------------- per-hit view ---------------- */
typedef struct { float x, y, z, r, zeta, rho, delta, T; } pt_t;

/* ---------------- cut predicates ---------------- */

/* Transverse bending of a hit pair a (inner) -> b (outer).  With u, v the components of
 * the step b - a across and along a's radial direction, a prompt track of radius
 * R >= Rmin has |u| / v <= T_b (T_b from the outer module's largest radius).  v is widened
 * by the radial tolerances; e adds the r-phi tolerance and the tangential shift a radial
 * error causes when a and b differ in phi.  The inequality |u| <= (v + rho) T + e is
 * evaluated multiplied by r_a > 0: U = u r_a, W = (v + rho) r_a, E = e r_a. */
static int pair_bend(const pt_t *a, const pt_t *b, float T) {
  float dx = b->x - a->x;
  float dy = b->y - a->y;
  float U = a->x * dy - a->y * dx;
  float V = a->x * dx + a->y * dy;
  float rs = a->rho + b->rho;
  float W = V + rs * a->r;
  float sphi = 0.0f; /* the radial-error term only exists when rs > 0 */
  if (rs != 0.0f) sphi = fabsf(a->x * b->y - a->y * b->x) / (a->r * b->r);
  float E = (C_E0 + rs * (sphi + 0.05f)) * a->r;
  return (W > 0.0f) && (fabsf(U) <= W * T + E);
}

/* r-z pointing of a hit pair: za rb - ra zb = z0 (rb - ra) for a straight line from
 * (0, z0); |z0| <= 15 cm, plus first-order resolution terms and the bound on the
 * arc-versus-radius difference of a curved track (no transcendental functions). */
static int pair_rz(const pt_t *a, const pt_t *b) {
  float f = a->z * b->r - a->r * b->z;
  float dr = fabsf(b->r - a->r);
  float dz = fabsf(b->z - a->z);
  float tol = C_Z0MAX * dr + (a->zeta * b->r + b->zeta * a->r + a->rho * fabsf(b->z) + b->rho * fabsf(a->z)) +
              C_KARC * dz * a->r * b->r * (a->r + b->r);
  return fabsf(f) <= tol;
}

/* Direction of an MD (upper minus lower hit, d) against the chord c of an LS that starts
 * or ends at that MD.  On a circle of radius R the tangent and a chord of length |c| make
 * an angle asin(|c| / 2R), so |d x c| <= |d| |c| (|c| / 2 Rmin) plus the error of d across
 * c.  No beam-line assumption: displaced tracks pass. */
static int md_dir(const pt_t *lo, const pt_t *up, float cx, float cy, float clen) {
  float dx = up->x - lo->x;
  float dy = up->y - lo->y;
  float dlen = sqrtf(dx * dx + dy * dy);
  float crs = fabsf(dx * cy - dy * cx);
  float tol = clen * (dlen * clen * C_HINV + C_EDIR + (lo->rho + up->rho));
  return crs <= tol;
}

/* Barrel-to-disk LS: the track must leave the barrel (|z| = zb_half) before it reaches
 * the next barrel layer, otherwise that layer is the next surface it crosses.  The r-z
 * line through the anchors exits at r_exit; the true track exits at a larger radius
 * (r grows more slowly than arc length), so r_exit <= r_next (+ resolution) never
 * rejects a track that does skip the layer. */
static int exit_ok(const pt_t *a, const pt_t *b, float rnext, float zb_half) {
  float Zb = b->z > 0.0f ? zb_half : -zb_half;
  float dzab = b->z - a->z;
  float t = (Zb - a->z) / dzab;
  float rexit = a->r + (b->r - a->r) * t;
  float ez = fabsf(Zb - b->z);
  float tol = rnext + b->rho + 0.5f + a->zeta * fabsf(b->r - a->r) * ez / (dzab * dzab);
  return rexit <= tol;
}

/* LS selection (reading of Sec. 1): pair bending and r-z pointing of the two anchors,
 * for barrel-to-disk pairs the barrel exit, and both MDs' directions consistent with the
 * chord. */
static int ls_pass(const pt_t *a, const pt_t *au, const pt_t *b, const pt_t *bu, float TB, float rnext_a,
                   int barrel_to_disk, float zb_half) {
  if (!(pair_bend(a, b, TB) && pair_rz(a, b))) return 0;
  if (barrel_to_disk && !exit_ok(a, b, rnext_a, zb_half)) return 0;
  float cx = b->x - a->x;
  float cy = b->y - a->y;
  float clen = sqrtf(cx * cx + cy * cy);
  return md_dir(a, au, cx, cy, clen) && md_dir(b, bu, cx, cy, clen);
}

/* r-z straightness of three hits p, q, s along the transverse chord: z is linear in arc
 * length, so (zq - zp) d_ps = (zs - zp) d_pq up to the arc/chord bound and the
 * resolution terms.  No beam-line constraint (displaced tracks). */
static void rz3_terms(const pt_t *p, const pt_t *q, const pt_t *s, float *lhs, float *tol) {
  float dxq = q->x - p->x, dyq = q->y - p->y;
  float dxs = s->x - p->x, dys = s->y - p->y;
  float dpq = sqrtf(dxq * dxq + dyq * dyq);
  float dps = sqrtf(dxs * dxs + dys * dys);
  float zqp = q->z - p->z;
  float zsp = s->z - p->z;
  *lhs = fabsf(zqp * dps - zsp * dpq);
  *tol = C_KARC * dps * dps * fabsf(zsp) * dpq + p->zeta * fabsf(dps - dpq) + q->zeta * dps + s->zeta * dpq +
         (p->rho + s->rho) * fabsf(zqp) + (p->rho + q->rho) * fabsf(zsp);
}

static int rz3(const pt_t *p, const pt_t *q, const pt_t *s) {
  float lhs, tol;
  rz3_terms(p, q, s, &lhs, &tol);
  return lhs <= tol;
}

static float max3f(float a, float b, float c) {
  float m = a > b ? a : b;
  return m > c ? m : c;
}

/* Signed curvature of the circle through p, q, s (coordinates centred at q):
 * k = 2 ((p - q) x (s - q)) / (|pq| |qs| |sp|); tol = 8 delta / |sp|^2 is the curvature
 * change a sagitta error delta causes. */
static void curv3(const pt_t *p, const pt_t *q, const pt_t *s, float *k, float *tol, float *cross_out,
                  float *prod_out, float *dsp_out) {
  float ax = p->x - q->x, ay = p->y - q->y;
  float cx = s->x - q->x, cy = s->y - q->y;
  float cross = ax * cy - ay * cx;
  float dpq = sqrtf(ax * ax + ay * ay);
  float dqs = sqrtf(cx * cx + cy * cy);
  float ex = s->x - p->x, ey = s->y - p->y;
  float dsp = sqrtf(ex * ex + ey * ey);
  float prod = dpq * dqs * dsp;
  float dmax = max3f(p->delta, q->delta, s->delta);
  *k = 2.0f * cross / prod;
  *tol = 8.0f * dmax / (dsp * dsp);
  if (cross_out) *cross_out = cross;
  if (prod_out) *prod_out = prod;
  if (dsp_out) *dsp_out = dpq + dqs + dsp;
}

/* Direction of the middle MD of a triple against the chord a -> c: on a circle the
 * tangent at b and the chord ac differ by half the difference of the arcs ab and bc, so
 * |d x ac| <= |d| |ac| ((|bc| - |ab|) + 2 % |ac|) / (2 Rmin) plus the error of d. */
static int mid_dir(const pt_t *a, const pt_t *b, const pt_t *bu, const pt_t *c) {
  float cx = c->x - a->x;
  float cy = c->y - a->y;
  float clen = sqrtf(cx * cx + cy * cy);
  float abx = b->x - a->x, aby = b->y - a->y;
  float bcx = c->x - b->x, bcy = c->y - b->y;
  float dab = sqrtf(abx * abx + aby * aby);
  float dbc = sqrtf(bcx * bcx + bcy * bcy);
  float dx = bu->x - b->x;
  float dy = bu->y - b->y;
  float dlen = sqrtf(dx * dx + dy * dy);
  float crs = fabsf(dx * cy - dy * cx);
  float tol = clen * (dlen * (fabsf(dbc - dab) + 0.02f * clen) * C_HINV + C_EDIR + (b->rho + bu->rho));
  return crs <= tol;
}

/* Circle radius of a triple: R = |ab||bc||ca| / (2 |cross|) >= Rmin (1 - 5 %), with the
 * cross product reduced by the point tolerance times the perimeter.  Straight triples pass. */
static int t3_radius(const pt_t *a, const pt_t *b, const pt_t *c) {
  float k, tol, cross, prod, perim;
  curv3(a, b, c, &k, &tol, &cross, &prod, &perim);
  float dmax = max3f(a->delta, b->delta, c->delta);
  float slack = fabsf(cross) - dmax * perim;
  return (slack <= 0.0f) || (prod >= C_K3 * slack);
}

/* T3 (Sec. 1: two LSs sharing an MD): r-z straightness, the middle MD's direction, and
 * a circle radius R = |ab||bc||ca| / (2 |cross|) >= Rmin (1 - 5 %) with the cross product
 * reduced by the point tolerance.  Straight triples pass. */
static int t3_pass(const pt_t *a, const pt_t *b, const pt_t *bu, const pt_t *c) {
  if (!rz3(a, b, c)) return 0;
  if (!mid_dir(a, b, bu, c)) return 0;
  return t3_radius(a, b, c);
}

/* The four circles of a T5 (a..e): inner (a,b,c), outer (c,d,e), bridge (b,c,d) and full
 * (a,c,e), their curvature differences d1 = |kin - kout|, d2 = |kbr - kfu| and the
 * right-hand sides of the two agreement conditions,
 * rhs = kappa (|k1| + |k2|) + tol1 + tol2 + kappa0. */
typedef struct { float kin, tin, kout, tout, kbr, tbr, kfu, tfu, d1, d2, rhs1, rhs2; } t5_circles;

static void t5_circles_of(const pt_t *P[5], t5_circles *c) {
  curv3(P[0], P[1], P[2], &c->kin, &c->tin, NULL, NULL, NULL);
  curv3(P[2], P[3], P[4], &c->kout, &c->tout, NULL, NULL, NULL);
  curv3(P[1], P[2], P[3], &c->kbr, &c->tbr, NULL, NULL, NULL);
  curv3(P[0], P[2], P[4], &c->kfu, &c->tfu, NULL, NULL, NULL);
  c->d1 = fabsf(c->kin - c->kout);
  c->d2 = fabsf(c->kbr - c->kfu);
  c->rhs1 = C_KAPPA * (fabsf(c->kin) + fabsf(c->kout)) + c->tin + c->tout + C_KAPPA0;
  c->rhs2 = C_KAPPA * (fabsf(c->kbr) + fabsf(c->kfu)) + c->tbr + c->tfu + C_KAPPA0;
}

/* x / (x + y) for non-negative x, y (0 when both are 0). */
static float frac_of(float x, float y) {
  float den = x + y;
  return den > 0.0f ? x / den : 0.0f;
}

/* Inputs of the learned T5 selection (Sec. 1 cites machine-learning methods among the LST
 * selections; this reading scores the curvature agreement with a small network instead of
 * the two kappa conditions).  Every input but f5 is a ratio x / (x + y) of non-negative
 * terms, so it lies in [0, 1):
 *   f0 = d1 / (d1 + rhs1)                 inner/outer difference against its tolerance
 *   f1 = d2 / (d2 + rhs2)                 bridge/full difference against its tolerance
 *   f2 = d1 / (d1 + |kin| + |kout| + kappa0)   relative inner/outer difference
 *   f3 = d2 / (d2 + |kbr| + |kfu| + kappa0)    relative bridge/full difference
 *   f4 = e / (e + |kin| + |kout| + kappa0), e = tol_in + tol_out: relative curvature error
 *   f5 = |kfu| / kmax                     full curvature against the pT threshold's
 *   f6 = l / (l + t), the r-z straightness residual l and tolerance t of (a, c, e)
 *   f7 = the same for (b, c, d), the triple across the shared MD c. */
static void t5_features_of(const pt_t *P[5], const t5_circles *c, float f[ORA_T5_NF]) {
  float l, t;
  f[0] = frac_of(c->d1, c->rhs1);
  f[1] = frac_of(c->d2, c->rhs2);
  f[2] = frac_of(c->d1, fabsf(c->kin) + fabsf(c->kout) + C_KAPPA0);
  f[3] = frac_of(c->d2, fabsf(c->kbr) + fabsf(c->kfu) + C_KAPPA0);
  f[4] = frac_of(c->tin + c->tout, fabsf(c->kin) + fabsf(c->kout) + C_KAPPA0);
  f[5] = fabsf(c->kfu) / C_KMAX;
  rz3_terms(P[0], P[2], P[4], &l, &t);
  f[6] = frac_of(l, t);
  rz3_terms(P[1], P[2], P[3], &l, &t);
  f[7] = frac_of(l, t);
}

/* The network: two hidden layers of ORA_T5_NH rectified units and a linear output,
 *   h1[j] = max(0, b1[j] + sum_i w1[j][i] f[i]),  h2[k] = max(0, b2[k] + sum_j w2[k][j] h1[j]),
 *   z = b3 + sum_k w3[k] h2[k],
 * in binary32, every sum accumulated from the bias in index order.  Weights in that order:
 * w1 (row j holds unit j's ORA_T5_NF inputs), b1, w2 (row k), b2, w3, b3.  The candidate
 * passes when z > 0. */
static float t5_mlp_logit(const float *w, const float f[ORA_T5_NF]) {
  const float *w1 = w, *b1 = w1 + ORA_T5_NH * ORA_T5_NF, *w2 = b1 + ORA_T5_NH;
  const float *b2 = w2 + ORA_T5_NH * ORA_T5_NH, *w3 = b2 + ORA_T5_NH, *b3 = w3 + ORA_T5_NH;
  float h1[ORA_T5_NH], h2[ORA_T5_NH];
  for (int j = 0; j < ORA_T5_NH; j++) {
    float a = b1[j];
    for (int i = 0; i < ORA_T5_NF; i++) a = a + w1[j * ORA_T5_NF + i] * f[i];
    h1[j] = a > 0.0f ? a : 0.0f;
  }
  for (int k = 0; k < ORA_T5_NH; k++) {
    float a = b2[k];
    for (int j = 0; j < ORA_T5_NH; j++) a = a + w2[k * ORA_T5_NH + j] * h1[j];
    h2[k] = a > 0.0f ? a : 0.0f;
  }
  float z = b3[0];
  for (int k = 0; k < ORA_T5_NH; k++) z = z + w3[k] * h2[k];
  return z;
}

/* T5 (Sec. 1: two T3s sharing an MD; circle-radius consistency): curvatures of the
 * inner (a,b,c), outer (c,d,e), bridge (b,c,d) and full (a,c,e) triples must agree,
 * the full circle must satisfy R >= Rmin (1 - 5 %), and a, c, e must be straight in r-z.
 * Returns the four conditions as bits 0-3 (inner/outer, bridge/full, radius, r-z).  With a
 * learned selection (mlp != NULL) the network's decision replaces both agreement
 * conditions: bits 0 and 1 are each z > 0. */
static unsigned t5_eval(const pt_t *P[5], const float *mlp, float *score, float *kfull_out) {
  t5_circles c;
  t5_circles_of(P, &c);
  int c1 = c.d1 <= c.rhs1;
  int c2 = c.d2 <= c.rhs2;
  int c3 = fabsf(c.kfu) <= C_KMAX + c.tfu;
  int c4 = rz3(P[0], P[2], P[4]);
  if (mlp) {
    float f[ORA_T5_NF];
    t5_features_of(P, &c, f);
    c1 = c2 = t5_mlp_logit(mlp, f) > 0.0f;
  }
  *score = c.d1 + c.d2;
  *kfull_out = c.kfu;
  return (unsigned)c1 | (unsigned)c2 << 1 | (unsigned)c3 << 2 | (unsigned)c4 << 3;
}

static int t5_pass(const pt_t *P[5], const float *mlp, float *score, float *kfull_out) {
  return t5_eval(P, mlp, score, kfull_out) == 15u;
}

/* ---------------- pLS helix and module lookup ---------------- */
typedef struct { float x0, y0, z0, R, cx, cy, cot, q, pt; int valid; } pls_t;

static void pls_params(const ora_pls *s, pls_t *o) {
  o->pt = sqrtf(s->px * s->px + s->py * s->py);
  o->R = o->pt / C_KB;
  float ux = s->px / o->pt;
  float uy = s->py / o->pt;
  o->q = (float)s->charge;
  float qR = o->q * o->R;
  o->x0 = s->x0; o->y0 = s->y0; o->z0 = s->z0;
  o->cx = s->x0 + qR * uy;
  o->cy = s->y0 - qR * ux;
  o->cot = s->pz / o->pt;
  o->valid = o->pt > 0.0f;
}

/* Arc length of a chord c on a circle of radius R: s = 2 R asin(c / 2R), with asin from
 * two half-angle reductions (sin(t/2) = x / sqrt(2 (1 + sqrt(1 - x^2)))) and the Taylor
 * series of asin to x^9; only + - * / sqrt. */
static float arc_len(float chord, float R) {
  float x = chord / (2.0f * R);
  if (x > 1.0f) x = 1.0f;
  float x1 = x / sqrtf(2.0f * (1.0f + sqrtf(1.0f - x * x)));
  float x2 = x1 / sqrtf(2.0f * (1.0f + sqrtf(1.0f - x1 * x1)));
  float t = x2 * x2;
  float as = x2 * (1.0f + t * (0.16666667f + t * (0.075f + t * (0.044642857f + t * 0.030381944f))));
  return 8.0f * R * as;
}

/* sin and cos of a in [0, pi]: Taylor series at a/4, then two angle doublings. */
static void sincos_series(float a, float *s_out, float *c_out) {
  float h = 0.25f * a;
  float h2 = h * h;
  float s = h * (1.0f - h2 / 6.0f * (1.0f - h2 / 20.0f * (1.0f - h2 / 42.0f * (1.0f - h2 / 72.0f * (1.0f - h2 / 110.0f)))));
  float c = 1.0f - h2 / 2.0f * (1.0f - h2 / 12.0f * (1.0f - h2 / 30.0f * (1.0f - h2 / 56.0f * (1.0f - h2 / 90.0f * (1.0f - h2 / 132.0f)))));
  float s2 = 2.0f * s * c;
  float c2 = c * c - s * s;
  *s_out = 2.0f * s2 * c2;
  *c_out = c2 * c2 - s2 * s2;
}

/* Sector of a ring row whose wedge holds direction (px, py): cross(e_k, P) >= 0 and
 * cross(e_{k+1}, P) < 0.  Returns -1 if none. */
static int find_sector(const ora_geom *g, int s, uint32_t row, float px, float py) {
  uint32_t n = g->row_nphi[s][row];
  for (uint32_t k = 0; k < n; k++) {
    uint32_t id = g->row_mod[s][row][k];
    if (id == UINT32_MAX) continue;
    const ora_module *m = &g->m[id];
    float c0 = m->e0x * py - m->e0y * px;
    float c1 = m->e1x * py - m->e1y * px;
    if (c0 >= 0.0f && c1 < 0.0f) return (int)k;
  }
  return -1;
}

static void add_cand(uint32_t *list, uint32_t *n, uint32_t id) {
  if (id == UINT32_MAX) return;
  for (uint32_t i = 0; i < *n; i++)
    if (list[i] == id) return;
  list[(*n)++] = id;
}

static void add_row_cands(const ora_geom *g, int s, int row, float px, float py, uint32_t *list, uint32_t *n) {
  if (row < 0 || (uint32_t)row >= g->n_rows[s] || !g->row_mod[s][row]) return;
  int k = find_sector(g, s, (uint32_t)row, px, py);
  if (k < 0) return;
  int nphi = (int)g->row_nphi[s][row];
  for (int d = -1; d <= 1; d++) {
    int kk = ((k + d) % nphi + nphi) % nphi;
    add_cand(list, n, g->row_mod[s][row][kk]);
  }
}

/* Candidate modules of a pLS (reading of "T3s and T5s are combined with IT tracks", Sec. 1):
 * extrapolate the pLS helix to barrel layers 1-2 (circle-circle intersection, first
 * crossing within half a turn) and to disks 1-2 on the side pz points to; each crossing
 * point selects its module and the neighbours +-1 in phi and in z (barrel) or ring
 * (endcap).  Up to 36 ids, sorted ascending. */
static uint32_t pls_candidates(const ora_geom *g, const pls_t *p, uint32_t out[36]) {
  uint32_t n = 0;
  if (!p->valid) return 0;
  for (int s = 0; s < 2; s++) {
    if (!g->n_rows[s]) continue;
    uint32_t any = g->surf_list[s][0];
    float rl = g->m[any].surf;
    float d2 = p->cx * p->cx + p->cy * p->cy;
    float d = sqrtf(d2);
    float a = (rl * rl - p->R * p->R + d2) / (2.0f * d);
    float h2 = rl * rl - a * a;
    if (!(h2 >= 0.0f)) continue;
    float h = sqrtf(h2);
    float ex = p->cx / d, ey = p->cy / d;
    float P1x = a * ex - h * ey, P1y = a * ey + h * ex;
    float P2x = a * ex + h * ey, P2y = a * ey - h * ex;
    float wx = p->x0 - p->cx, wy = p->y0 - p->cy;
    float cr1 = wx * (P1y - p->cy) - wy * (P1x - p->cx);
    float cr2 = wx * (P2y - p->cy) - wy * (P2x - p->cx);
    int f1 = -p->q * cr1 > 0.0f;
    int f2 = -p->q * cr2 > 0.0f;
    float dt1 = wx * (P1x - p->cx) + wy * (P1y - p->cy);
    float dt2 = wx * (P2x - p->cx) + wy * (P2y - p->cy);
    float Px, Py;
    if (f1 && f2) {
      if (dt1 >= dt2) { Px = P1x; Py = P1y; } else { Px = P2x; Py = P2y; }
    } else if (f1) {
      Px = P1x; Py = P1y;
    } else if (f2) {
      Px = P2x; Py = P2y;
    } else {
      continue;
    }
    float dxc = Px - p->x0, dyc = Py - p->y0;
    float chord = sqrtf(dxc * dxc + dyc * dyc);
    float sarc = arc_len(chord, p->R);
    float zP = p->z0 + sarc * p->cot;
    /* z bins: row 0 starts at emin, rows are (emax - emin) long */
    if (!g->row_mod[s][0] || g->row_mod[s][0][0] == UINT32_MAX) continue;
    const ora_module *m0 = &g->m[g->row_mod[s][0][0]];
    float zlen = m0->emax - m0->emin;
    float zhi = m0->emin + (float)g->n_rows[s] * zlen;
    if (!(zP > m0->emin - 2.0f * zlen && zP < zhi + 2.0f * zlen)) continue;
    int iz = (int)floorf((zP - m0->emin) / zlen);
    for (int dz = -1; dz <= 1; dz++) add_row_cands(g, s, iz + dz, Px, Py, out, &n);
  }
  if (p->cot != 0.0f) {
    int side0 = p->cot > 0.0f ? 11 : 6;
    for (int di = 0; di < 2; di++) {
      int s = side0 + di;
      if (!g->n_rows[s] || !g->row_mod[s][0] || g->row_mod[s][0][0] == UINT32_MAX) continue;
      const ora_module *m0 = &g->m[g->row_mod[s][0][0]];
      float zd = m0->surf;
      float sarc = (zd - p->z0) / p->cot;
      if (!(sarc > 0.0f)) continue;
      float alpha = sarc / p->R;
      if (!(alpha < C_PI)) continue;
      float sa, ca;
      sincos_series(alpha, &sa, &ca);
      float sn = -p->q * sa;
      float wx = p->x0 - p->cx, wy = p->y0 - p->cy;
      float Px = p->cx + (wx * ca - wy * sn);
      float Py = p->cy + (wx * sn + wy * ca);
      float rP = sqrtf(Px * Px + Py * Py);
      float rlen = m0->emax - m0->emin;
      float rhi = m0->emin + (float)g->n_rows[s] * rlen;
      if (!(rP > m0->emin - 2.0f * rlen && rP < rhi + 2.0f * rlen)) continue;
      int ir = (int)floorf((rP - m0->emin) / rlen);
      for (int dr = -1; dr <= 1; dr++) add_row_cands(g, s, ir + dr, Px, Py, out, &n);
    }
  }
  qsort(out, n, sizeof(uint32_t), cmp_u32);
  return n;
}

/* pLS-to-anchor compatibility (reading of pT3/pT5, Sec. 1): each anchor must lie within
 * an r-phi window of the pLS circle and an r-z window of the pLS line, both growing with
 * the arc length s from the reference point (1 % pT, 1 mrad phi and direction spread).
 * Adds the normalised squared residuals to *score; returns the r-phi (bit 0) and r-z
 * (bit 1) window decisions. */
static unsigned pls_anchor_eval(const pls_t *p, const pt_t *X, float *score) {
  float ddx = X->x - p->x0, ddy = X->y - p->y0;
  float chord = sqrtf(ddx * ddx + ddy * ddy);
  float s = arc_len(chord, p->R);
  float ex = X->x - p->cx, ey = X->y - p->cy;
  float dphi = sqrtf(ex * ex + ey * ey) - p->R;
  float wphi = C_W0 + 0.003f * s + 0.015f * s * s / p->R + X->rho;
  float ez = X->z - (p->z0 + s * p->cot);
  float wz = 0.05f + 0.002f * s + X->zeta + X->rho * fabsf(p->cot);
  float a = dphi / wphi, b = ez / wz;
  *score = *score + (a * a + b * b);
  return (unsigned)(fabsf(dphi) <= wphi) | (unsigned)(fabsf(ez) <= wz) << 1;
}

static int pls_anchor(const pls_t *p, const pt_t *X, float *score) { return pls_anchor_eval(p, X, score) == 3u; }

/* pT5 (reading of Sec. 1): the T5's full-circle curvature must agree with the pLS's,
 * ||k_full| - 1/R| <= 15 % / R plus the curvature tolerance of the T5's (a, c, e) triple. */
static int pt5_curv(const pls_t *p, float kf, const pt_t *P0, const pt_t *P2, const pt_t *P4) {
  float kk, tf;
  curv3(P0, P2, P4, &kk, &tf, NULL, NULL, NULL);
  return fabsf(fabsf(kf) - 1.0f / p->R) <= C_KPT5 / p->R + tf;
}

/* Pseudo-angle of (x, y) in [0, 4): 0 along +x, 1 along +y, 2 along -x, 3 along -y,
 * increasing with the azimuth inside each quadrant (y / (x + y) in the first), from
 * divisions only, so that binary32 gives the same value everywhere.  The origin maps to 0.
 * Hits of one sensor are ordered by it (reading of "objects sorted", R17: azimuth order
 * inside a module). */
static float pseudo_angle(float x, float y) {
  if (y >= 0.0f) {
    if (x >= 0.0f) {
      float den = x + y;
      return den > 0.0f ? y / den : 0.0f;
    }
    return 1.0f + (-x) / (y - x);
  }
  if (x < 0.0f) return 2.0f + (-y) / (-x - y);
  return 3.0f + x / (x - y);
}

/* ---------------- the chain ---------------- */
typedef struct {
  const ora_geom *g;
  pt_t *hit;
  uint32_t *md_off; /* per module */
  vu32 md_module, md_lo, md_up;
} ctx_t;

static void get_pt(const ora_geom *g, const ora_event *ev, uint32_t h, uint32_t module, pt_t *o) {
  o->x = ev->x[h]; o->y = ev->y[h]; o->z = ev->z[h];
  o->r = sqrtf(o->x * o->x + o->y * o->y);
  o->zeta = g->zeta[module]; o->rho = g->rho[module]; o->delta = g->delta[module]; o->T = g->T[module];
}

static int count_shared(const uint32_t *a, int na, const uint32_t *b, int nb) {
  int c = 0;
  for (int i = 0; i < na; i++)
    for (int j = 0; j < nb; j++)
      if (a[i] == b[j]) c++;
  return c;
}

/* MD -> objects inverse lists (CSR) for duplicate search. */
static int build_md_index(uint32_t n_md, const uint32_t *mds, uint32_t n_obj, int per, uint32_t **off_out,
                          uint32_t **list_out) {
  uint32_t *off = (uint32_t *)calloc(n_md + 1, sizeof(uint32_t));
  if (!off) return -1;
  for (uint32_t o = 0; o < n_obj; o++)
    for (int k = 0; k < per; k++) off[mds[(size_t)o * per + k] + 1]++;
  for (uint32_t i = 0; i < n_md; i++) off[i + 1] += off[i];
  uint32_t *cur = (uint32_t *)malloc((n_md + 1) * sizeof(uint32_t));
  uint32_t *list = (uint32_t *)malloc(((size_t)off[n_md] + 1) * sizeof(uint32_t));
  if (!cur || !list) { free(off); free(cur); free(list); return -1; }
  memcpy(cur, off, (n_md + 1) * sizeof(uint32_t));
  for (uint32_t o = 0; o < n_obj; o++)
    for (int k = 0; k < per; k++) list[cur[mds[(size_t)o * per + k]]++] = o;
  free(cur);
  *off_out = off;
  *list_out = list;
  return 0;
}

static int better(float sy, uint32_t y, float sx, uint32_t x) { return sy < sx || (sy == sx && y < x); }

int ora_run(const ora_geom *g, const ora_event *ev, int brute_ls, ora_result *out) {
  memset(out, 0, sizeof(*out));
  int rc = -1;
  uint32_t nh = ev->n_hits, nm = g->n;
  pt_t *hit = NULL;
  uint32_t *bin_off = NULL, *bin_list = NULL, *md_off = NULL, *ls_off = NULL, *t3_off = NULL, *t5_off = NULL;
  uint32_t *idx5 = NULL, *lst5 = NULL, *idx3 = NULL, *lst3 = NULL, *idxt = NULL, *lstt = NULL;
  uint8_t *used5 = NULL, *used3 = NULL, *cross3 = NULL, *crosst = NULL;
  uint32_t *pls_md3 = NULL, *pls_md5 = NULL;
  pls_t *pl = NULL;
  vu32 md_module = {0}, md_lo = {0}, md_up = {0}, ls = {0}, t3 = {0}, t5 = {0};
  vf32 t5s = {0}, t5k = {0};
  vu32 pt3p = {0}, pt3o = {0}, pt5p = {0}, pt5o = {0};
  vf32 pt3s = {0}, pt5s = {0};

  for (uint32_t i = 0; i < nh; i++) {
    if (ev->det[i] >= 2u * nm) goto done;
    if (!isfinite(ev->x[i]) || !isfinite(ev->y[i]) || !isfinite(ev->z[i])) goto done;
  }
  for (uint32_t p = 0; p < ev->n_pls; p++)
    if (ev->pls[p].n_hits != 0 && ev->pls[p].n_hits != 3 && ev->pls[p].n_hits != 4) goto done;
  /* ---- hit binning by module sensor, in azimuth order inside each sensor (pseudo-angle,
   * ties by input index) ---- */
  bin_off = (uint32_t *)calloc(2 * (size_t)nm + 1, sizeof(uint32_t));
  bin_list = (uint32_t *)malloc(((size_t)nh + 1) * sizeof(uint32_t));
  hit = (pt_t *)malloc(((size_t)nh + 1) * sizeof(pt_t));
  if (!bin_off || !bin_list || !hit) goto done;
  for (uint32_t i = 0; i < nh; i++) bin_off[ev->det[i] + 1]++;
  for (uint32_t i = 0; i < 2 * nm; i++) bin_off[i + 1] += bin_off[i];
  {
    uint32_t *cur = (uint32_t *)malloc((2 * (size_t)nm + 1) * sizeof(uint32_t));
    if (!cur) goto done;
    memcpy(cur, bin_off, (2 * (size_t)nm + 1) * sizeof(uint32_t));
    for (uint32_t i = 0; i < nh; i++) bin_list[cur[ev->det[i]]++] = i;
    free(cur);
  }
  {
    float *psi = (float *)malloc(((size_t)nh + 1) * sizeof(float));
    if (!psi) goto done;
    for (uint32_t i = 0; i < nh; i++) psi[i] = pseudo_angle(ev->x[i], ev->y[i]);
    for (uint32_t s = 0; s < 2 * nm; s++) /* insertion sort: sensors hold a few hits */
      for (uint32_t i = bin_off[s] + 1; i < bin_off[s + 1]; i++) {
        uint32_t h = bin_list[i], j = i;
        while (j > bin_off[s] && (psi[bin_list[j - 1]] > psi[h] ||
                                  (psi[bin_list[j - 1]] == psi[h] && bin_list[j - 1] > h))) {
          bin_list[j] = bin_list[j - 1];
          j--;
        }
        bin_list[j] = h;
      }
    free(psi);
  }
  for (uint32_t i = 0; i < nh; i++) get_pt(g, ev, i, ev->det[i] >> 1, &hit[i]);

  /* ---- Mini Doublets: every lower x upper hit pair of a module (Sec. 1) ---- */
  md_off = (uint32_t *)malloc(((size_t)nm + 1) * sizeof(uint32_t));
  if (!md_off) goto done;
  for (uint32_t m = 0; m < nm; m++) {
    md_off[m] = (uint32_t)md_lo.n;
    float T = g->T[m];
    for (uint32_t i = bin_off[2 * m]; i < bin_off[2 * m + 1]; i++) {
      uint32_t a = bin_list[i];
      for (uint32_t j = bin_off[2 * m + 1]; j < bin_off[2 * m + 2]; j++) {
        uint32_t b = bin_list[j];
        out->n_tests[0]++;
        if (pair_bend(&hit[a], &hit[b], T) && pair_rz(&hit[a], &hit[b])) {
          if (vu32_push(&md_module, m) || vu32_push(&md_lo, a) || vu32_push(&md_up, b)) goto done;
        }
      }
    }
  }
  md_off[nm] = (uint32_t)md_lo.n;
  uint32_t n_md = (uint32_t)md_lo.n;

  /* ---- Line Segments: MD on A x MD on B, B in the connection map of A (Sec. 1) ---- */
  ls_off = (uint32_t *)malloc(((size_t)n_md + 1) * sizeof(uint32_t));
  if (!ls_off) goto done;
  {
    uint32_t *brute_list = NULL;
    if (brute_ls) brute_list = (uint32_t *)malloc(((size_t)nm + 1) * sizeof(uint32_t));
    if (brute_ls && !brute_list) goto done;
    for (uint32_t a = 0; a < n_md; a++) {
      ls_off[a] = (uint32_t)(ls.n / 2);
      uint32_t A = md_module.p[a];
      const pt_t *pa = &hit[md_lo.p[a]], *pau = &hit[md_up.p[a]];
      const uint32_t *nb;
      uint32_t nnb;
      if (brute_ls) {
        int nxt[3];
        int k = next_surfaces(g->surface[A], nxt);
        nnb = 0;
        for (int t = 0; t < k; t++)
          for (uint32_t q = 0; q < g->surf_count[nxt[t]]; q++) brute_list[nnb++] = g->surf_list[nxt[t]][q];
        qsort(brute_list, nnb, sizeof(uint32_t), cmp_u32);
        nb = brute_list;
      } else {
        nb = g->cols + g->row_off[A];
        nnb = g->row_off[A + 1] - g->row_off[A];
      }
      for (uint32_t q = 0; q < nnb; q++) {
        uint32_t B = nb[q];
        float TB = g->T[B];
        int b2d = g->m[A].subdet == 0 && g->m[B].subdet == 1;
        for (uint32_t b = md_off[B]; b < md_off[B + 1]; b++) {
          out->n_tests[1]++;
          if (ls_pass(pa, pau, &hit[md_lo.p[b]], &hit[md_up.p[b]], TB, g->rnext[A], b2d, g->zb_half)) {
            if (vu32_push(&ls, a) || vu32_push(&ls, b)) { free(brute_list); goto done; }
          }
        }
      }
    }
    free(brute_list);
  }
  ls_off[n_md] = (uint32_t)(ls.n / 2);

  /* ---- T3: LS (a->b) + LS (b->c) sharing MD b (Sec. 1) ---- */
  t3_off = (uint32_t *)malloc(((size_t)n_md + 1) * sizeof(uint32_t));
  if (!t3_off) goto done;
  for (uint32_t a = 0; a < n_md; a++) {
    t3_off[a] = (uint32_t)(t3.n / 3);
    const pt_t *pa = &hit[md_lo.p[a]];
    for (uint32_t l1 = ls_off[a]; l1 < ls_off[a + 1]; l1++) {
      uint32_t b = ls.p[2 * l1 + 1];
      const pt_t *pb = &hit[md_lo.p[b]];
      for (uint32_t l2 = ls_off[b]; l2 < ls_off[b + 1]; l2++) {
        uint32_t c = ls.p[2 * l2 + 1];
        out->n_tests[2]++;
        if (t3_pass(pa, pb, &hit[md_up.p[b]], &hit[md_lo.p[c]])) {
          if (vu32_push(&t3, a) || vu32_push(&t3, b) || vu32_push(&t3, c)) goto done;
        }
      }
    }
  }
  t3_off[n_md] = (uint32_t)(t3.n / 3);

  /* ---- T5: T3 (a,b,c) + T3 (c,d,e) sharing MD c (Sec. 1) ---- */
  t5_off = (uint32_t *)malloc(((size_t)n_md + 1) * sizeof(uint32_t));
  if (!t5_off) goto done;
  for (uint32_t a = 0; a < n_md; a++) {
    t5_off[a] = (uint32_t)(t5.n / 5);
    for (uint32_t i1 = t3_off[a]; i1 < t3_off[a + 1]; i1++) {
      uint32_t b = t3.p[3 * i1 + 1], c = t3.p[3 * i1 + 2];
      for (uint32_t i2 = t3_off[c]; i2 < t3_off[c + 1]; i2++) {
        uint32_t d = t3.p[3 * i2 + 1], e = t3.p[3 * i2 + 2];
        const pt_t *P[5] = {&hit[md_lo.p[a]], &hit[md_lo.p[b]], &hit[md_lo.p[c]], &hit[md_lo.p[d]],
                            &hit[md_lo.p[e]]};
        float score, kf;
        out->n_tests[3]++;
        if (t5_pass(P, g->t5_mlp, &score, &kf)) {
          if (vu32_push(&t5, a) || vu32_push(&t5, b) || vu32_push(&t5, c) || vu32_push(&t5, d) ||
              vu32_push(&t5, e) || vf32_push(&t5s, score) || vf32_push(&t5k, kf))
            goto done;
        }
      }
    }
  }
  t5_off[n_md] = (uint32_t)(t5.n / 5);
  uint32_t n_t5 = t5_off[n_md], n_t3 = t3_off[n_md];

  /* ---- pLS: candidate modules, then pT3 and pT5 (Sec. 1) ---- */
  uint32_t np = ev->n_pls;
  out->pls_cand_n = (uint32_t *)calloc((size_t)np + 1, sizeof(uint32_t));
  out->pls_cand = (uint32_t *)calloc((size_t)np * 36 + 1, sizeof(uint32_t));
  pl = (pls_t *)malloc(((size_t)np + 1) * sizeof(pls_t));
  if (!out->pls_cand_n || !out->pls_cand || !pl) goto done;
  for (uint32_t p = 0; p < np; p++) {
    pls_params(&ev->pls[p], &pl[p]);
    out->n_tests[4]++;
    out->pls_cand_n[p] = pls_candidates(g, &pl[p], out->pls_cand + (size_t)p * 36);
  }
  for (uint32_t p = 0; p < np; p++) {
    for (uint32_t ci = 0; ci < out->pls_cand_n[p]; ci++) {
      uint32_t M = out->pls_cand[(size_t)p * 36 + ci];
      for (uint32_t a = md_off[M]; a < md_off[M + 1]; a++) {
        for (uint32_t t = t3_off[a]; t < t3_off[a + 1]; t++) {
          float score = 0.0f;
          int ok = 1;
          out->n_tests[5]++;
          for (int k = 0; k < 3; k++) ok &= pls_anchor(&pl[p], &hit[md_lo.p[t3.p[3 * t + k]]], &score);
          if (ok && (vu32_push(&pt3p, p) || vu32_push(&pt3o, t) || vf32_push(&pt3s, score))) goto done;
        }
      }
    }
  }
  for (uint32_t p = 0; p < np; p++) {
    for (uint32_t ci = 0; ci < out->pls_cand_n[p]; ci++) {
      uint32_t M = out->pls_cand[(size_t)p * 36 + ci];
      for (uint32_t a = md_off[M]; a < md_off[M + 1]; a++) {
        for (uint32_t t = t5_off[a]; t < t5_off[a + 1]; t++) {
          float score = 0.0f;
          int ok = 1;
          out->n_tests[6]++;
          for (int k = 0; k < 5; k++) ok &= pls_anchor(&pl[p], &hit[md_lo.p[t5.p[5 * t + k]]], &score);
          const pt_t *P0 = &hit[md_lo.p[t5.p[5 * t]]], *P2 = &hit[md_lo.p[t5.p[5 * t + 2]]],
                     *P4 = &hit[md_lo.p[t5.p[5 * t + 4]]];
          int c5 = pt5_curv(&pl[p], t5k.p[t], P0, P2, P4);
          if (ok && c5 && (vu32_push(&pt5p, p) || vu32_push(&pt5o, t) || vf32_push(&pt5s, score))) goto done;
        }
      }
    }
  }
  uint32_t n_pt3 = (uint32_t)pt3p.n, n_pt5 = (uint32_t)pt5p.n;

  /* ---- duplicate removal (reading of "only a subset is propagated", Sec. 1) ----
   * Stage order pT5 -> pT3 -> T5 -> pLS.  Inside a stage an object dies iff another
   * object of the same stage that survived the earlier stages' removal overlaps it and
   * ranks better (lower score, then lower index) -- one pass over the whole stage, so
   * the result does not depend on processing order.  Overlap: same pLS, or shared MDs
   * (pT5 >= 3, pT3 >= 2, T5 >= 3).  Across stages: a pT3 dies if its pLS is used by a
   * surviving pT5 or it shares >= 2 MDs with one; a T5 dies if it shares >= 3 MDs with
   * a surviving pT5 or pT3; a pLS is a TC iff no surviving pT3/pT5 uses it. */
  out->alive_pt5 = (uint8_t *)calloc((size_t)n_pt5 + 1, 1);
  out->alive_pt3 = (uint8_t *)calloc((size_t)n_pt3 + 1, 1);
  out->alive_t5 = (uint8_t *)calloc((size_t)n_t5 + 1, 1);
  out->pls_tc = (uint8_t *)calloc((size_t)np + 1, 1);
  used5 = (uint8_t *)calloc((size_t)np + 1, 1);
  used3 = (uint8_t *)calloc((size_t)np + 1, 1);
  cross3 = (uint8_t *)calloc((size_t)n_pt3 + 1, 1);
  crosst = (uint8_t *)calloc((size_t)n_t5 + 1, 1);
  pls_md5 = (uint32_t *)malloc(((size_t)n_pt5 * 5 + 1) * sizeof(uint32_t));
  pls_md3 = (uint32_t *)malloc(((size_t)n_pt3 * 3 + 1) * sizeof(uint32_t));
  if (!out->alive_pt5 || !out->alive_pt3 || !out->alive_t5 || !out->pls_tc || !used5 || !used3 || !cross3 ||
      !crosst || !pls_md5 || !pls_md3)
    goto done;
  for (uint32_t i = 0; i < n_pt5; i++)
    for (int k = 0; k < 5; k++) pls_md5[5 * i + k] = t5.p[5 * pt5o.p[i] + k];
  for (uint32_t i = 0; i < n_pt3; i++)
    for (int k = 0; k < 3; k++) pls_md3[3 * i + k] = t3.p[3 * pt3o.p[i] + k];
  if (build_md_index(n_md, pls_md5, n_pt5, 5, &idx5, &lst5)) goto done;
  if (build_md_index(n_md, pls_md3, n_pt3, 3, &idx3, &lst3)) goto done;
  if (build_md_index(n_md, t5.p, n_t5, 5, &idxt, &lstt)) goto done;
  /* pT5 stage */
  for (uint32_t x = 0; x < n_pt5; x++) {
    int dead = 0;
    for (uint32_t y = x; y-- > 0 && pt5p.p[y] == pt5p.p[x] && !dead;)
      if (better(pt5s.p[y], y, pt5s.p[x], x)) dead = 1;
    for (uint32_t y = x + 1; y < n_pt5 && pt5p.p[y] == pt5p.p[x] && !dead; y++)
      if (better(pt5s.p[y], y, pt5s.p[x], x)) dead = 1;
    for (int k = 0; k < 5 && !dead; k++) {
      uint32_t m = pls_md5[5 * x + k];
      for (uint32_t j = idx5[m]; j < idx5[m + 1] && !dead; j++) {
        uint32_t y = lst5[j];
        if (y == x) continue;
        if (count_shared(pls_md5 + 5 * x, 5, pls_md5 + 5 * y, 5) >= 3 && better(pt5s.p[y], y, pt5s.p[x], x)) dead = 1;
      }
    }
    out->alive_pt5[x] = !dead;
    if (!dead) used5[pt5p.p[x]] = 1;
  }
  /* pT3 stage */
  for (uint32_t x = 0; x < n_pt3; x++) {
    int dead = used5[pt3p.p[x]];
    for (int k = 0; k < 3 && !dead; k++) {
      uint32_t m = pls_md3[3 * x + k];
      for (uint32_t j = idx5[m]; j < idx5[m + 1] && !dead; j++) {
        uint32_t z = lst5[j];
        if (out->alive_pt5[z] && count_shared(pls_md3 + 3 * x, 3, pls_md5 + 5 * z, 5) >= 2) dead = 1;
      }
    }
    cross3[x] = (uint8_t)dead;
  }
  for (uint32_t x = 0; x < n_pt3; x++) {
    int dead = cross3[x];
    for (uint32_t y = x; y-- > 0 && pt3p.p[y] == pt3p.p[x] && !dead;)
      if (!cross3[y] && better(pt3s.p[y], y, pt3s.p[x], x)) dead = 1;
    for (uint32_t y = x + 1; y < n_pt3 && pt3p.p[y] == pt3p.p[x] && !dead; y++)
      if (!cross3[y] && better(pt3s.p[y], y, pt3s.p[x], x)) dead = 1;
    for (int k = 0; k < 3 && !dead; k++) {
      uint32_t m = pls_md3[3 * x + k];
      for (uint32_t j = idx3[m]; j < idx3[m + 1] && !dead; j++) {
        uint32_t y = lst3[j];
        if (y == x || cross3[y]) continue;
        if (count_shared(pls_md3 + 3 * x, 3, pls_md3 + 3 * y, 3) >= 2 && better(pt3s.p[y], y, pt3s.p[x], x)) dead = 1;
      }
    }
    out->alive_pt3[x] = !dead;
    if (!dead) used3[pt3p.p[x]] = 1;
  }
  /* T5 stage */
  for (uint32_t x = 0; x < n_t5; x++) {
    int dead = 0;
    const uint32_t *mx = t5.p + 5 * (size_t)x;
    for (int k = 0; k < 5 && !dead; k++) {
      uint32_t m = mx[k];
      for (uint32_t j = idx5[m]; j < idx5[m + 1] && !dead; j++) {
        uint32_t z = lst5[j];
        if (out->alive_pt5[z] && count_shared(mx, 5, pls_md5 + 5 * z, 5) >= 3) dead = 1;
      }
      for (uint32_t j = idx3[m]; j < idx3[m + 1] && !dead; j++) {
        uint32_t z = lst3[j];
        if (out->alive_pt3[z] && count_shared(mx, 5, pls_md3 + 3 * z, 3) >= 3) dead = 1;
      }
    }
    crosst[x] = (uint8_t)dead;
  }
  for (uint32_t x = 0; x < n_t5; x++) {
    int dead = crosst[x];
    const uint32_t *mx = t5.p + 5 * (size_t)x;
    for (int k = 0; k < 5 && !dead; k++) {
      uint32_t m = mx[k];
      for (uint32_t j = idxt[m]; j < idxt[m + 1] && !dead; j++) {
        uint32_t y = lstt[j];
        if (y == x || crosst[y]) continue;
        if (count_shared(mx, 5, t5.p + 5 * (size_t)y, 5) >= 3 && better(t5s.p[y], y, t5s.p[x], x)) dead = 1;
      }
    }
    out->alive_t5[x] = !dead;
  }
  for (uint32_t p = 0; p < np; p++) out->pls_tc[p] = !(used5[p] || used3[p]);

  /* ---- track candidates: pT5, pT3, T5, pLS (Sec. 1 list) ---- */
  {
    uint32_t ntc = 0;
    for (uint32_t x = 0; x < n_pt5; x++) ntc += out->alive_pt5[x];
    for (uint32_t x = 0; x < n_pt3; x++) ntc += out->alive_pt3[x];
    for (uint32_t x = 0; x < n_t5; x++) ntc += out->alive_t5[x];
    for (uint32_t p = 0; p < np; p++) ntc += out->pls_tc[p];
    out->n_tc = ntc;
    out->tc_type = (uint8_t *)malloc((size_t)ntc + 1);
    out->tc_obj = (uint32_t *)malloc(((size_t)ntc + 1) * sizeof(uint32_t));
    out->tc_pls = (uint32_t *)malloc(((size_t)ntc + 1) * sizeof(uint32_t));
    out->tc_ot = (uint32_t *)malloc(((size_t)ntc * 10 + 1) * sizeof(uint32_t));
    out->tc_pix = (uint32_t *)malloc(((size_t)ntc * 4 + 1) * sizeof(uint32_t));
    out->tc_pt = (float *)malloc(((size_t)ntc + 1) * sizeof(float));
    out->tc_score = (float *)malloc(((size_t)ntc + 1) * sizeof(float));
    if (!out->tc_type || !out->tc_obj || !out->tc_pls || !out->tc_ot || !out->tc_pix || !out->tc_pt || !out->tc_score)
      goto done;
    uint32_t w = 0;
    for (int type = 0; type < 4; type++) {
      uint32_t nobj = type == 0 ? n_pt5 : type == 1 ? n_pt3 : type == 2 ? n_t5 : np;
      for (uint32_t x = 0; x < nobj; x++) {
        const uint8_t *alive = type == 0 ? out->alive_pt5 : type == 1 ? out->alive_pt3 : type == 2 ? out->alive_t5 : out->pls_tc;
        if (!alive[x]) continue;
        uint32_t pls = UINT32_MAX, nmd = 0;
        const uint32_t *mds = NULL;
        float score = 0.0f, pt = 0.0f;
        if (type == 0) { pls = pt5p.p[x]; mds = pls_md5 + 5 * (size_t)x; nmd = 5; score = pt5s.p[x]; }
        if (type == 1) { pls = pt3p.p[x]; mds = pls_md3 + 3 * (size_t)x; nmd = 3; score = pt3s.p[x]; }
        if (type == 2) { mds = t5.p + 5 * (size_t)x; nmd = 5; score = t5s.p[x]; pt = C_KB / fabsf(t5k.p[x]); }
        if (type == 3) { pls = x; }
        if (pls != UINT32_MAX) pt = pl[pls].pt;
        out->tc_type[w] = (uint8_t)type;
        out->tc_obj[w] = x;
        out->tc_pls[w] = pls;
        for (int k = 0; k < 10; k++) out->tc_ot[10 * (size_t)w + k] = UINT32_MAX;
        for (uint32_t k = 0; k < nmd; k++) {
          out->tc_ot[10 * (size_t)w + 2 * k] = md_lo.p[mds[k]];
          out->tc_ot[10 * (size_t)w + 2 * k + 1] = md_up.p[mds[k]];
        }
        /* the seed's pixel hits: four for a quad, the first three for a triplet */
        uint32_t npix = pls == UINT32_MAX ? 0 : (ev->pls[pls].n_hits == 3 ? 3 : 4);
        for (uint32_t k = 0; k < 4; k++) out->tc_pix[4 * (size_t)w + k] = k < npix ? 4 * pls + k : UINT32_MAX;
        out->tc_pt[w] = pt;
        out->tc_score[w] = score;
        w++;
      }
    }
  }

  out->n_md = n_md; out->md_module = md_module.p; out->md_lo = md_lo.p; out->md_up = md_up.p;
  md_module.p = md_lo.p = md_up.p = NULL;
  out->n_ls = ls_off[n_md]; out->ls_md = ls.p; ls.p = NULL;
  out->n_t3 = n_t3; out->t3_md = t3.p; t3.p = NULL;
  out->n_t5 = n_t5; out->t5_md = t5.p; out->t5_score = t5s.p; out->t5_kfull = t5k.p;
  t5.p = NULL; t5s.p = t5k.p = NULL;
  out->n_pt3 = n_pt3; out->pt3_pls = pt3p.p; out->pt3_obj = pt3o.p; out->pt3_score = pt3s.p;
  pt3p.p = pt3o.p = NULL; pt3s.p = NULL;
  out->n_pt5 = n_pt5; out->pt5_pls = pt5p.p; out->pt5_obj = pt5o.p; out->pt5_score = pt5s.p;
  pt5p.p = pt5o.p = NULL; pt5s.p = NULL;
  rc = 0;
done:
  free(hit); free(bin_off); free(bin_list); free(md_off); free(ls_off); free(t3_off); free(t5_off);
  free(idx5); free(lst5); free(idx3); free(lst3); free(idxt); free(lstt);
  free(used5); free(used3); free(cross3); free(crosst); free(pls_md3); free(pls_md5); free(pl);
  free(md_module.p); free(md_lo.p); free(md_up.p); free(ls.p); free(t3.p); free(t5.p); free(t5s.p); free(t5k.p);
  free(pt3p.p); free(pt3o.p); free(pt3s.p); free(pt5p.p); free(pt5o.p); free(pt5s.p);
  if (rc) ora_result_free(out);
  return rc;
}

void ora_result_free(ora_result *r) {
  if (!r) return;
  free(r->md_module); free(r->md_lo); free(r->md_up); free(r->ls_md); free(r->t3_md);
  free(r->t5_md); free(r->t5_score); free(r->t5_kfull);
  free(r->pt3_pls); free(r->pt3_obj); free(r->pt3_score);
  free(r->pt5_pls); free(r->pt5_obj); free(r->pt5_score);
  free(r->pls_cand_n); free(r->pls_cand);
  free(r->alive_pt5); free(r->alive_pt3); free(r->alive_t5); free(r->pls_tc);
  free(r->tc_type); free(r->tc_obj); free(r->tc_pls); free(r->tc_ot); free(r->tc_pix);
  free(r->tc_pt); free(r->tc_score);
  memset(r, 0, sizeof(*r));
}

/* ---------------- event-parallel driver (for CPU timing only) ---------------- */
typedef struct {
  const ora_geom *g;
  const ora_event *evs;
  ora_result *outs;
  uint32_t n, next;
  int rc;
  pthread_mutex_t mu;
} pool_t;

static void *worker(void *arg) {
  pool_t *p = (pool_t *)arg;
  for (;;) {
    pthread_mutex_lock(&p->mu);
    uint32_t i = p->next++;
    pthread_mutex_unlock(&p->mu);
    if (i >= p->n) break;
    if (ora_run(p->g, &p->evs[i], 0, &p->outs[i])) {
      pthread_mutex_lock(&p->mu);
      p->rc = -1;
      pthread_mutex_unlock(&p->mu);
    }
  }
  return NULL;
}

int ora_run_many(const ora_geom *g, const ora_event *evs, uint32_t n, int n_threads, ora_result *outs) {
  pool_t p = {g, evs, outs, n, 0, 0, PTHREAD_MUTEX_INITIALIZER};
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < n_threads; t++)
    if (pthread_create(&th[t], NULL, worker, &p) == 0) started++;
  if (!started) worker(&p);
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  return p.rc;
}

/* ---------------- exported helpers, for pinning the oracle in tests ---------------- */
float ora_arc_len(float chord, float R) { return arc_len(chord, R); }
void ora_sincos(float a, float *s, float *c) { sincos_series(a, s, c); }
int ora_md_test(const ora_geom *g, uint32_t module, const float a[3], const float b[3]) {
  pt_t pa, pb;
  pa.x = a[0]; pa.y = a[1]; pa.z = a[2]; pa.r = sqrtf(pa.x * pa.x + pa.y * pa.y);
  pb.x = b[0]; pb.y = b[1]; pb.z = b[2]; pb.r = sqrtf(pb.x * pb.x + pb.y * pb.y);
  pa.zeta = pb.zeta = g->zeta[module];
  pa.rho = pb.rho = g->rho[module];
  pa.delta = pb.delta = g->delta[module];
  pa.T = pb.T = g->T[module];
  return pair_bend(&pa, &pb, g->T[module]) && pair_rz(&pa, &pb);
}

/* Predicate-level evaluation, so that tests can show which single condition a
 * constructed configuration fails.  Points are (x, y, z); each takes the tolerances of
 * the module given beside it.  Every function only calls the predicates the chain uses. */
static void load_pt(const ora_geom *g, uint32_t module, const float v[3], pt_t *o) {
  o->x = v[0]; o->y = v[1]; o->z = v[2];
  o->r = sqrtf(o->x * o->x + o->y * o->y);
  o->zeta = g->zeta[module]; o->rho = g->rho[module]; o->delta = g->delta[module]; o->T = g->T[module];
}

uint32_t ora_ls_eval(const ora_geom *g, uint32_t A, uint32_t B, const float a[3], const float au[3],
                     const float b[3], const float bu[3]) {
  if (A >= g->n || B >= g->n) return 0;
  pt_t pa, pau, pb, pbu;
  load_pt(g, A, a, &pa); load_pt(g, A, au, &pau); load_pt(g, B, b, &pb); load_pt(g, B, bu, &pbu);
  int b2d = g->m[A].subdet == 0 && g->m[B].subdet == 1;
  float cx = pb.x - pa.x;
  float cy = pb.y - pa.y;
  float clen = sqrtf(cx * cx + cy * cy);
  uint32_t m = 0;
  m |= (uint32_t)pair_bend(&pa, &pb, g->T[B]);
  m |= (uint32_t)pair_rz(&pa, &pb) << 1;
  m |= (uint32_t)(!b2d || exit_ok(&pa, &pb, g->rnext[A], g->zb_half)) << 2;
  m |= (uint32_t)md_dir(&pa, &pau, cx, cy, clen) << 3;
  m |= (uint32_t)md_dir(&pb, &pbu, cx, cy, clen) << 4;
  return m;
}

uint32_t ora_t3_eval(const ora_geom *g, const uint32_t mod[3], const float a[3], const float b[3],
                     const float bu[3], const float c[3]) {
  for (int k = 0; k < 3; k++)
    if (mod[k] >= g->n) return 0;
  pt_t pa, pb, pbu, pc;
  load_pt(g, mod[0], a, &pa); load_pt(g, mod[1], b, &pb); load_pt(g, mod[1], bu, &pbu); load_pt(g, mod[2], c, &pc);
  return (uint32_t)rz3(&pa, &pb, &pc) | (uint32_t)mid_dir(&pa, &pb, &pbu, &pc) << 1 |
         (uint32_t)t3_radius(&pa, &pb, &pc) << 2;
}

uint32_t ora_t5_eval(const ora_geom *g, const uint32_t mod[5], const float p[15], float *score, float *kfull) {
  pt_t q[5];
  const pt_t *P[5];
  for (int k = 0; k < 5; k++) {
    if (mod[k] >= g->n) return 0;
    load_pt(g, mod[k], p + 3 * k, &q[k]);
    P[k] = &q[k];
  }
  return t5_eval(P, g->t5_mlp, score, kfull);
}

uint32_t ora_t5_features(const ora_geom *g, const uint32_t mod[5], const float p[15], float f[ORA_T5_NF]) {
  pt_t q[5];
  const pt_t *P[5];
  for (int k = 0; k < 5; k++) {
    if (mod[k] >= g->n) return 0;
    load_pt(g, mod[k], p + 3 * k, &q[k]);
    P[k] = &q[k];
  }
  t5_circles c;
  t5_circles_of(P, &c);
  t5_features_of(P, &c, f);
  return 1;
}

float ora_t5_logit(const float *w, const float f[ORA_T5_NF]) { return t5_mlp_logit(w, f); }

int ora_geom_set_t5_mlp(ora_geom *g, const float *w, uint32_t n) {
  if (!w) {
    free(g->t5_mlp);
    g->t5_mlp = NULL;
    return 0;
  }
  if (n != ORA_T5_NPARAM) return -1;
  for (uint32_t i = 0; i < n; i++)
    if (!isfinite(w[i])) return -1;
  float *c = (float *)malloc(n * sizeof(float));
  if (!c) return -1;
  memcpy(c, w, n * sizeof(float));
  free(g->t5_mlp);
  g->t5_mlp = c;
  return 0;
}

uint32_t ora_pls_eval(const ora_geom *g, const ora_pls *s, uint32_t module, const float x[3], float *score) {
  if (module >= g->n) return 0;
  pls_t p;
  pt_t X;
  pls_params(s, &p);
  load_pt(g, module, x, &X);
  *score = 0.0f;
  return pls_anchor_eval(&p, &X, score);
}

/* bit 0: all five anchors inside the pLS windows; bit 1: the pT5 curvature agreement. */
uint32_t ora_pt5_eval(const ora_geom *g, const ora_pls *s, const uint32_t mod[5], const float pts[15]) {
  pt_t q[5];
  const pt_t *P[5];
  pls_t p;
  pls_params(s, &p);
  for (int k = 0; k < 5; k++) {
    if (mod[k] >= g->n) return 0;
    load_pt(g, mod[k], pts + 3 * k, &q[k]);
    P[k] = &q[k];
  }
  float score = 0.0f, t5score, kf;
  int ok = 1;
  for (int k = 0; k < 5; k++) ok &= pls_anchor(&p, P[k], &score);
  t5_eval(P, NULL, &t5score, &kf);
  return (uint32_t)ok | (uint32_t)pt5_curv(&p, kf, P[0], P[2], P[4]) << 1;
}
