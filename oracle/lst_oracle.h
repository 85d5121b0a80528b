/*
 * CPU oracle for the Line Segment Tracking hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C (FP32 arithmetic, no contraction, no fast math) that
 * computes the object sets the method defines: Mini-Doublets (MD), Line Segments (LS),
 * T3, T5, pLS-module lookup, pT3, pT5, duplicate removal and track candidates (TC).
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may use it; the
 * CUDA library never links or calls it and shares no code with it.
 *
 * The paper (Sec. 1) names the objects and the order they are built in, but prints no
 * cut: every numeric selection here is this project's stated reading, written out in
 * lst_oracle.c beside the step it belongs to.
 *
 * Record layouts mirror the detector-description and pixel-seed records of the input
 * generator (48-byte module, 80-byte seed).
 */
#ifndef LST_ORACLE_H
#define LST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint8_t subdet;  /* 0 barrel, 1 endcap */
  uint8_t layer;   /* barrel layer 1..6, endcap disk 1..5 */
  int8_t side;     /* 0 barrel, -1/+1 endcap */
  uint8_t stype;   /* 0 PS, 1 2S */
  uint16_t ieta;   /* barrel z bin, endcap ring */
  uint16_t iphi;
  uint16_t nphi;
  uint16_t pad;
  float surf;      /* barrel: lower-sensor radius; endcap: lower-sensor signed z */
  float gap;       /* sensor separation */
  float emin, emax;/* barrel: z extent; endcap: r extent */
  float e0x, e0y;  /* lower phi edge (unit vector) */
  float e1x, e1y;  /* upper phi edge (unit vector) */
  float tilt;      /* barrel: tilt of the module in the r-z plane (rad), 0 = flat; endcap: 0 */
} ora_module;

typedef struct {
  float px, py, pz;   /* momentum at the reference point (GeV) */
  float x0, y0, z0;   /* reference point (cm) */
  float hx[4], hy[4], hz[4]; /* pixel hits (a triplet: the first three) */
  int32_t charge;     /* +1 / -1 */
  uint32_t n_hits;    /* pixel hits: 4 (quad; 0 is read as 4) or 3 (triplet) */
} ora_pls;

typedef struct {
  uint32_t n_hits;
  const float *x, *y, *z;
  const uint32_t *det; /* 2 * module + sensor */
  uint32_t n_pls;
  const ora_pls *pls;
} ora_event;

enum { ORA_TC_PT5 = 0, ORA_TC_PT3 = 1, ORA_TC_T5 = 2, ORA_TC_PLS = 3 };

typedef struct {
  uint32_t n_md;  uint32_t *md_module, *md_lo, *md_up;   /* lo/up = input hit indices */
  uint32_t n_ls;  uint32_t *ls_md;                       /* 2 MD indices per LS */
  uint32_t n_t3;  uint32_t *t3_md;                       /* 3 per T3 */
  uint32_t n_t5;  uint32_t *t5_md; float *t5_score, *t5_kfull; /* 5 per T5 */
  uint32_t n_pt3; uint32_t *pt3_pls, *pt3_obj; float *pt3_score;
  uint32_t n_pt5; uint32_t *pt5_pls, *pt5_obj; float *pt5_score;
  uint32_t *pls_cand_n, *pls_cand; /* per pLS: candidate-module count and up to 36 ids */
  uint8_t *alive_pt5, *alive_pt3, *alive_t5, *pls_tc;
  uint32_t n_tc;
  uint8_t *tc_type; uint32_t *tc_obj, *tc_pls, *tc_ot /*10 per*/, *tc_pix /*4 per*/;
  float *tc_pt, *tc_score;
  uint64_t n_tests[7]; /* candidate tests: MD, LS, T3, T5, pLS-module, pT3, pT5 */
} ora_result;

typedef struct ora_geom ora_geom;

/* Copies the module table, derives the per-module cut constants and builds the module
 * connection map.  Returns NULL on bad input. */
ora_geom *ora_geom_create(const ora_module *mods, uint32_t n_mods);
void ora_geom_destroy(ora_geom *g);
/* Connection map as CSR: row_off has n_mods+1 entries; returns the number of edges. */
uint32_t ora_geom_map(const ora_geom *g, const uint32_t **row_off, const uint32_t **cols);

/* Runs the whole chain on one event.  brute_ls != 0 ignores the connection map and tests
 * every MD pair on adjacent surfaces (used to check that the map loses nothing).
 * Returns 0 on success. */
int ora_run(const ora_geom *g, const ora_event *ev, int brute_ls, ora_result *out);
void ora_result_free(ora_result *r);

/* Runs ora_run over n events on up to n_threads threads (events are independent). */
int ora_run_many(const ora_geom *g, const ora_event *evs, uint32_t n, int n_threads,
                 ora_result *outs);

/* Helpers exported only so tests can pin them against library routines. */
float ora_arc_len(float chord, float R);
void ora_sincos(float a, float *s, float *c);
int ora_md_test(const ora_geom *g, uint32_t module, const float a[3], const float b[3]);
/* Predicate-level decisions as bit masks (tests only).  LS: bending, r-z pointing, barrel
 * exit (1 unless barrel to disk), inner-MD direction, outer-MD direction.  T3: r-z
 * straightness, middle-MD direction, radius.  T5: inner/outer curvature, bridge/full
 * curvature, full radius, (a, c, e) r-z straightness (also returns score and k_full).
 * pLS anchor: r-phi window, r-z window.  pT5: all five anchor windows, curvature. */
uint32_t ora_ls_eval(const ora_geom *g, uint32_t A, uint32_t B, const float a[3], const float au[3],
                     const float b[3], const float bu[3]);
uint32_t ora_t3_eval(const ora_geom *g, const uint32_t mod[3], const float a[3], const float b[3],
                     const float bu[3], const float c[3]);
uint32_t ora_t5_eval(const ora_geom *g, const uint32_t mod[5], const float p[15], float *score, float *kfull);

/* Learned T5 selection: ORA_T5_NF inputs per candidate, two hidden layers of ORA_T5_NH
 * units, ORA_T5_NPARAM weights (w1, b1, w2, b2, w3, b3; see t5_mlp_logit).
 * ora_geom_set_t5_mlp copies the weights into the geometry (w == NULL: back to the kappa
 * cuts); returns 0, or -1 when n != ORA_T5_NPARAM or a weight is not finite.
 * ora_t5_features fills f (returns 0 when a module id is out of range);
 * ora_t5_logit evaluates the network on f. */
#define ORA_T5_NF 8
#define ORA_T5_NH 16
#define ORA_T5_NPARAM (ORA_T5_NH * ORA_T5_NF + ORA_T5_NH + ORA_T5_NH * ORA_T5_NH + ORA_T5_NH + ORA_T5_NH + 1)
int ora_geom_set_t5_mlp(ora_geom *g, const float *w, uint32_t n);
uint32_t ora_t5_features(const ora_geom *g, const uint32_t mod[5], const float p[15], float f[ORA_T5_NF]);
float ora_t5_logit(const float *w, const float f[ORA_T5_NF]);
uint32_t ora_pls_eval(const ora_geom *g, const ora_pls *s, uint32_t module, const float x[3], float *score);
uint32_t ora_pt5_eval(const ora_geom *g, const ora_pls *s, const uint32_t mod[5], const float pts[15]);

#ifdef __cplusplus
}
#endif
#endif
