// Device-side data views shared by the kernels and the host runtime of liblst.
#pragma once
#include <cstdint>

#include "lst_cuts.cuh"

namespace lst {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int NSURF = 16;
constexpr int MAX_CAND = 36;
constexpr uint32_t LS_LIST_MAX = 2048;  // longest neighbour list the LS count pass stages
constexpr uint32_t PLS_MD_CAP = 64;  // MDs passing a pLS's first-anchor test, kept per pLS
// pT3 items of one pLS: its kept MDs, or (more passing MDs) its candidate modules
constexpr uint32_t PLS_ITEMS = PLS_MD_CAP > (uint32_t)MAX_CAND ? PLS_MD_CAP : (uint32_t)MAX_CAND;

constexpr int N_SCAN_SLOTS = 16;          // scans of one run that can take the single-pass form
constexpr uint32_t SCAN_LARGE_CHUNK = 8192; // elements per block of a large single-pass scan

// Totals written by the scans into the batch header.
enum Total : int {
  T_HITS = 0, T_MD, T_LS, T_T3, T_T5, T_PT3, T_PT5, T_C5, T_C3, T_CT, T_A5, T_A3, T_AT, T_AP, T_TC, T_PT3I, N_TOTALS
};
constexpr uint32_t ERR_BAD_INPUT = 1u;
constexpr uint32_t ERR_WAIT = 2u;  // a bounded device-side wait ran out (the run is discarded)
constexpr uint32_t ERR_OVERFLOW_SHIFT = 8;  // bit (8 + Total) = that list outgrew its storage

// pLS record as the device reads it (layout of lst_pls).
struct PlsIn {
  float px, py, pz, x0, y0, z0;
  float hx[4], hy[4], hz[4];
  int32_t charge;
  uint32_t n_hits;  // pixel hits: 4 (quad; 0 is read as 4) or 3 (triplet)
};

// Per-batch header in device memory: input pointers, sizes, totals, error word.
struct Hdr {
  const float *x, *y, *z;
  const uint32_t *det, *hit_off;
  const PlsIn *pls;
  const uint32_t *pls_off;
  uint32_t n_ev, n_hits, n_pls, pad;
  uint32_t tot[N_TOTALS];
  uint32_t err;
  uint32_t ls_maxlen;  // LS count pass: the longest neighbour list beyond the launch's list cap
  uint32_t scan_epoch;  // this run's number (1, 2, ...): tags the chunk states of the large scans
  uint32_t pad2;
  uint32_t mask_used[8];  // LS partner-list arena: [1] words handed out in pieces (may pass the
                          // arena's end), [2] words of the lists that found it exhausted
  unsigned long long ls_cand;  // MD pairs the LS count pass tested (connection-map candidates)
  uint32_t work[16];           // work counters of the dynamically scheduled kernels (W_*)
  // single-pass scans: per scan, the ticket counter that hands out its chunks in block start
  // order (the chunk states themselves are in BufView::scan_state)
  uint32_t scan_ticket[N_SCAN_SLOTS];
};

// Work counters in Hdr::work, one per dynamically scheduled kernel and pass.
enum WorkCounter : int { W_LS = 0, W_PT3_COUNT, W_PT5_COUNT, W_PT3_FIRST, W_MD, N_WORK };
static_assert(N_WORK <= 16, "Hdr::work too small");

// Geometry tables (device pointers) and per-geometry scalars.
struct GeoView {
  uint32_t nm;
  float zb_half;
  const float4 *modc;   // zeta, rho, delta, T
  const float *rnext;   // next barrel layer radius (1e30 if none)
  const uint8_t *subdet;
  const uint32_t *conn_off, *conn;
  const float* conn_dpsi;  // per map edge: pseudo-angle half-width of the LS bending window
  const float4 *mod_e;  // e0x, e0y, e1x, e1y
  const float4 *mod_g;  // surf, gap, emin, emax
  int32_t surf_first[NSURF];
  uint32_t surf_nrows[NSURF];
  uint32_t surf_row_base[NSURF];
  const uint32_t *row_nphi, *row_mod_base, *row_mods;
  // rows whose wedges partition the circle (every sector present, each upper edge equal
  // bit for bit to the next sector's lower edge): at most one sector can hold a point, so a
  // guessed sector checked with the exact test gives the linear scan's answer
  const uint8_t *row_fast;
  const float *row_phi0;  // angle of sector 0's lower edge
};

// Pipeline buffers (device pointers) and capacities.
struct BufView {
  Hdr *hdr;
  uint32_t cap_ev, cap_hits, cap_md, cap_ls, cap_t3, cap_t5, cap_pls, cap_pt3, cap_pt5, cap_tc;
  // hits
  uint32_t *sen_cnt, *sen_off, *hit_tmp, *hit_ev, *hit_idx;
  float *hit_psi;     // pseudo-angle of the hit at the same position of hit_tmp
  uint32_t *hit_sen;  // per sorted hit: its sensor bucket (event * 2 modules + sensor)
  float4 *hit4;
  // MD
  uint32_t *md_hcnt, *md_hoff;  // per sorted hit: MDs with it as the lower hit, their offset
  uint32_t *md_hmask;          // per sorted lower hit: pass bits of its first 32 candidates
  uint32_t *md_off, *md_unit, *md_lo_idx, *md_up_idx;
  float4 *md_pt;  // per MD, one 32-byte sector: [2m] lower hit (x, y, z, r), [2m + 1] module tolerances
  float4 *md_up4;
  float4 *md_dir4;  // upper - lower hit: dx, dy, transverse length, rho + rho
  float *md_psi;    // pseudo-angle of the lower hit (a module's MDs are in its order)
  float4 *md_box;   // per unit: its MDs' lower-hit box, (x0, x1, y0, y1), (z0, z1, -, -)
  // LS
  uint32_t *ls_cnt, *ls_off, *ls_in, *ls_out;
  // T3: per LS count/offset of the T3s built on it, per MD offset of those starting there
  uint32_t *t3_lcnt, *t3_loff, *t3_off, *t3_a, *t3_b, *t3_c;
  uint32_t *t3_mask;  // per LS: pass bits of its first 32 candidates (count pass -> fill pass)
  uint4 *t3_md4;      // per T3: (a, b, c, 0), one load for duplicate removal
  // T5: per T3 count/offset of the T5s built on it, per MD offset
  uint32_t *t5_tcnt, *t5_toff, *t5_off, *t5_m0, *t5_m1, *t5_m2, *t5_m3, *t5_m4;
  uint32_t *t5_mask;  // per T3: pass bits of its first 32 candidates
  uint4 *t5_md8;      // per T5: (m0, m1, m2, m3), (m4, 0, 0, 0), two loads for duplicate removal
  float *t5_score, *t5_kfull;
  // pLS
  uint32_t *pls_ev, *pls_ncand, *pls_cand;
  uint32_t *pls_mdpass, *pls_nmdpass;  // MDs passing the first-anchor test (64 per pLS; NONE: more)
  float4 *pls_h0, *pls_h1;  // (x0, y0, z0, R), (cx, cy, cot, q)
  float *pls_pt;
  // pT3 / pT5
  uint32_t *pt3_icnt, *pt3_ioff;  // per pLS: pT3 items (phase-2 MDs, or candidate modules), offsets
  uint32_t *pt3_item_p;          // per item: its pLS
  uint32_t *pt3_xcnt, *pt3_xoff, *pt3_xmask;  // per item: pT3s, their offset, pass bits
  uint32_t *pt3_off, *pt3_pls, *pt3_obj;
  float *pt3_score;
  uint32_t *pt5_xcnt, *pt5_xoff, *pt5_xmask;  // per pT3: pT5s on it, their offset, pass bits
  uint32_t *pt5_off, *pt5_pls, *pt5_obj;
  float *pt5_score;
  // duplicate removal: MD -> object lists and flags (u32 so they can be scanned)
  uint32_t *c5_cnt, *c5_off, *c5_list, *c3_cnt, *c3_off, *c3_list, *ct_cnt, *ct_off, *ct_list;
  uint32_t *alive5, *alive3, *alivet, *plstc, *cross3, *crosst;
  uint32_t *sa5, *sa3, *sat, *sap;  // exclusive scans of the alive flags
  // track candidates
  uint32_t *tc_ev_off;
  void *tc;  // lst_tc records
  // join scratch: chunk ballots of the count passes, and each unit's slice of them
  // scratch arena: the LS count pass's partner lists [count, partner MDs] (mask_off: per
  // anchor MD its list's offset, or NONE when the fill pass must join it again)
  uint32_t *mask, *mask_off;
  uint32_t cap_mask;
  // single-pass scans of large arrays: scan_chunks chunk states per scan slot (null where no
  // scan is large)
  unsigned long long* scan_state;
  uint32_t scan_chunks;
};

typedef void (*MarkFn)(void* arg, int kernel_name);
extern const char* const kKernelNames[];
extern const int kNumKernelNames;

// A second stream for the pLS side of the chain: the pLS preparation (needs only the inputs)
// forked at the start, then pT3 phase 1 once the MDs exist; joined before the pT3 count, so
// it overlaps the hit, MD, LS, T3 and T5 stages.  Null: one stream.
struct SideBranch {
  cudaStream_t s;
  cudaEvent_t fork, mds, join;  // chain start; MDs written; side work done
};

struct Launch {
  uint32_t grid;   // persistent grid (blocks)
  uint32_t block;  // threads per block
  uint32_t ls_list_cap;  // LS: neighbour MDs staged per warp (0: per-MD join everywhere)
  const T5Mlp* t5_mlp = nullptr;  // learned T5 selection (host copy, passed by value), null: the cuts
};

}  // namespace lst
