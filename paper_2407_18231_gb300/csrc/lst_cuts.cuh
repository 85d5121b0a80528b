// Selection arithmetic of the LST chain, device side.
//
// Every predicate is IEEE binary32 with + - * / sqrtf fabsf and comparisons only, compiled
// with --fmad=false -prec-div=true -prec-sqrt=true -ftz=false, and every expression keeps
// one fixed evaluation order, so the results are reproducible bit for bit.  Points are
// float4 (x, y, z, r = sqrtf(x*x + y*y)); a point's module tolerances come as float4
// (zeta: z, rho: radial, delta: transverse, T: bending slope of the module).
//
// The paper (arXiv:2407.18231, Sec. 1) defines the objects (MD, LS, T3, T5, pT3, pT5) and
// the order they are built in but prints no cut; the selections here are this project's
// reading, derived from helix geometry: a prompt track of curvature radius R >= Rmin
// (pT >= 0.8 GeV at 3.8 T) crosses radius r at an angle asin(r / 2R) to the radial
// direction, and its z grows linearly with arc length.
#pragma once
#include <cstdint>

namespace lst {

struct MethodConst {
  float KB;      // pT [GeV] per cm of curvature radius (0.0029979 * 3.8)
  float Z0MAX;   // luminous-region half length used for r-z pointing (cm)
  float E0;      // r-phi tolerance of a hit pair (cm)
  float KARC;    // bound on (arc - chord) effects: 2 / (24 Rmin^2)
  float K3;      // 2 Rmin (1 - 5 %)
  float KMAX;    // largest accepted curvature 1 / (Rmin (1 - 5 %))
  float KAPPA;   // relative curvature agreement of T5 sub-triples
  float KAPPA0;  // absolute curvature slack (1/cm)
  float KPT5;    // pT5: T5 versus pLS curvature (relative)
  float W0;      // pLS r-phi window floor (cm)
  float PI;
  float HINV;    // 1 / (2 Rmin): sine of the tangent-chord angle per cm of chord
  float EDIR;    // error of an MD direction across a chord (cm)
};

struct PointTol {
  float4 p;  // x, y, z, r
  float4 t;  // zeta, rho, delta, T
};

// Transverse bending of a hit pair a (inner) -> b (outer): the step's component across
// a's radial direction (u) against its radial component (v), |u| <= v T + e, evaluated
// multiplied through by r_a (U = u r_a, W = (v + rho) r_a) so that no division is needed
// unless a hit has a radial tolerance (endcap).
__device__ __forceinline__ bool pair_bend(const MethodConst& C, const PointTol& a, const PointTol& b, float T) {
  const float dx = b.p.x - a.p.x;
  const float dy = b.p.y - a.p.y;
  const float U = a.p.x * dy - a.p.y * dx;
  const float V = a.p.x * dx + a.p.y * dy;
  const float rs = a.t.y + b.t.y;
  const float W = V + rs * a.p.w;
  float sphi = 0.0f;  // rs * (sphi + 0.05) below is +0 when rs == 0, whatever sphi is
  if (rs != 0.0f) sphi = fabsf(a.p.x * b.p.y - a.p.y * b.p.x) / (a.p.w * b.p.w);
  const float E = (C.E0 + rs * (sphi + 0.05f)) * a.p.w;
  return (W > 0.0f) && (fabsf(U) <= W * T + E);
}

// r-z pointing of a hit pair: za rb - ra zb = z0 (rb - ra) for a line from (0, z0).
__device__ __forceinline__ bool pair_rz(const MethodConst& C, const PointTol& a, const PointTol& b) {
  const float f = a.p.z * b.p.w - a.p.w * b.p.z;
  const float dr = fabsf(b.p.w - a.p.w);
  const float dz = fabsf(b.p.z - a.p.z);
  const float tol = C.Z0MAX * dr + (a.t.x * b.p.w + b.t.x * a.p.w + a.t.y * fabsf(b.p.z) + b.t.y * fabsf(a.p.z)) +
                    C.KARC * dz * a.p.w * b.p.w * (a.p.w + b.p.w);
  return fabsf(f) <= tol;
}

// Direction of an MD (upper minus lower hit) against a chord c that starts or ends at it:
// tangent and chord of length |c| differ by asin(|c| / 2R).
__device__ __forceinline__ bool md_dir(const MethodConst& C, const PointTol& lo, const PointTol& up, float cx, float cy,
                                       float clen) {
  const float dx = up.p.x - lo.p.x;
  const float dy = up.p.y - lo.p.y;
  const float dlen = sqrtf(dx * dx + dy * dy);
  const float crs = fabsf(dx * cy - dy * cx);
  const float tol = clen * (dlen * clen * C.HINV + C.EDIR + (lo.t.y + up.t.y));
  return crs <= tol;
}

// The MD half of md_dir, for an MD whose direction terms were stored by md_direction:
// the same operations in the same order, so the same decision bit for bit.
__device__ __forceinline__ float4 md_direction(const float4& lo, const float4& up, const float4& cst) {
  const float dx = up.x - lo.x;
  const float dy = up.y - lo.y;
  return make_float4(dx, dy, sqrtf(dx * dx + dy * dy), cst.y + cst.y);
}
__device__ __forceinline__ bool md_dir_pre(const MethodConst& C, const float4& d, float cx, float cy, float clen) {
  const float crs = fabsf(d.x * cy - d.y * cx);
  const float tol = clen * (d.z * clen * C.HINV + C.EDIR + d.w);
  return crs <= tol;
}

// Barrel-to-disk LS: the anchors' r-z line must leave the barrel before the next layer.
__device__ __forceinline__ bool exit_ok(const PointTol& a, const PointTol& b, float rnext, float zb_half) {
  const float Zb = b.p.z > 0.0f ? zb_half : -zb_half;
  const float dzab = b.p.z - a.p.z;
  const float t = (Zb - a.p.z) / dzab;
  const float rexit = a.p.w + (b.p.w - a.p.w) * t;
  const float ez = fabsf(Zb - b.p.z);
  const float tol = rnext + b.t.y + 0.5f + a.t.x * fabsf(b.p.w - a.p.w) * ez / (dzab * dzab);
  return rexit <= tol;
}

__device__ __forceinline__ bool ls_select(const MethodConst& C, const PointTol& a, const PointTol& au, const PointTol& b,
                                          const PointTol& bu, float rnext_a, bool barrel_to_disk, float zb_half) {
  if (!(pair_rz(C, a, b) && pair_bend(C, a, b, b.t.w))) return false;  // cheaper test first
  if (barrel_to_disk && !exit_ok(a, b, rnext_a, zb_half)) return false;
  const float cx = b.p.x - a.p.x;
  const float cy = b.p.y - a.p.y;
  const float clen = sqrtf(cx * cx + cy * cy);
  return md_dir(C, a, au, cx, cy, clen) && md_dir(C, b, bu, cx, cy, clen);
}

// r-z straightness of p, q, s along the transverse chord (z linear in arc length): the
// residual lhs and its tolerance; the triple is straight when lhs <= tol.
__device__ __forceinline__ void rz3_terms(const MethodConst& C, const PointTol& p, const PointTol& q,
                                          const PointTol& s, float& lhs, float& tol) {
  const float dxq = q.p.x - p.p.x, dyq = q.p.y - p.p.y;
  const float dxs = s.p.x - p.p.x, dys = s.p.y - p.p.y;
  const float dpq = sqrtf(dxq * dxq + dyq * dyq);
  const float dps = sqrtf(dxs * dxs + dys * dys);
  const float zqp = q.p.z - p.p.z;
  const float zsp = s.p.z - p.p.z;
  lhs = fabsf(zqp * dps - zsp * dpq);
  tol = C.KARC * dps * dps * fabsf(zsp) * dpq + p.t.x * fabsf(dps - dpq) + q.t.x * dps + s.t.x * dpq +
        (p.t.y + s.t.y) * fabsf(zqp) + (p.t.y + q.t.y) * fabsf(zsp);
}

__device__ __forceinline__ bool rz3(const MethodConst& C, const PointTol& p, const PointTol& q, const PointTol& s) {
  float lhs, tol;
  rz3_terms(C, p, q, s, lhs, tol);
  return lhs <= tol;
}

// Middle MD direction against chord a -> c (inscribed-angle relation).
__device__ __forceinline__ bool mid_dir(const MethodConst& C, const PointTol& a, const PointTol& b, const PointTol& bu,
                                        const PointTol& c) {
  const float cx = c.p.x - a.p.x;
  const float cy = c.p.y - a.p.y;
  const float clen = sqrtf(cx * cx + cy * cy);
  const float abx = b.p.x - a.p.x, aby = b.p.y - a.p.y;
  const float bcx = c.p.x - b.p.x, bcy = c.p.y - b.p.y;
  const float dab = sqrtf(abx * abx + aby * aby);
  const float dbc = sqrtf(bcx * bcx + bcy * bcy);
  const float dx = bu.p.x - b.p.x;
  const float dy = bu.p.y - b.p.y;
  const float dlen = sqrtf(dx * dx + dy * dy);
  const float crs = fabsf(dx * cy - dy * cx);
  const float tol = clen * (dlen * (fabsf(dbc - dab) + 0.02f * clen) * C.HINV + C.EDIR + (b.t.y + bu.t.y));
  return crs <= tol;
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  const float m = a > b ? a : b;
  return m > c ? m : c;
}

struct Circle3 {
  float k, tol, cross, prod, perim;
};

// Signed curvature of the circle through p, q, s, centred at q.
__device__ __forceinline__ Circle3 circle3(const PointTol& p, const PointTol& q, const PointTol& s) {
  const float ax = p.p.x - q.p.x, ay = p.p.y - q.p.y;
  const float cx = s.p.x - q.p.x, cy = s.p.y - q.p.y;
  const float cross = ax * cy - ay * cx;
  const float dpq = sqrtf(ax * ax + ay * ay);
  const float dqs = sqrtf(cx * cx + cy * cy);
  const float ex = s.p.x - p.p.x, ey = s.p.y - p.p.y;
  const float dsp = sqrtf(ex * ex + ey * ey);
  const float prod = dpq * dqs * dsp;
  const float dmax = max3(p.t.z, q.t.z, s.t.z);
  Circle3 r;
  r.k = 2.0f * cross / prod;
  r.tol = 8.0f * dmax / (dsp * dsp);
  r.cross = cross;
  r.prod = prod;
  r.perim = dpq + dqs + dsp;
  return r;
}

__device__ __forceinline__ bool t3_select(const MethodConst& C, const PointTol& a, const PointTol& b, const PointTol& bu,
                                          const PointTol& c) {
  if (!rz3(C, a, b, c)) return false;
  if (!mid_dir(C, a, b, bu, c)) return false;
  const Circle3 k = circle3(a, b, c);
  const float dmax = max3(a.t.z, b.t.z, c.t.z);
  const float slack = fabsf(k.cross) - dmax * k.perim;
  return (slack <= 0.0f) || (k.prod >= C.K3 * slack);
}

__device__ __forceinline__ bool t5_select(const MethodConst& C, const PointTol& A, const PointTol& B, const PointTol& Cc,
                                          const PointTol& D, const PointTol& E, float& score, float& kfull) {
  const Circle3 in = circle3(A, B, Cc);
  const Circle3 out = circle3(Cc, D, E);
  const Circle3 br = circle3(B, Cc, D);
  const Circle3 fu = circle3(A, Cc, E);
  const float d1 = fabsf(in.k - out.k);
  const float d2 = fabsf(br.k - fu.k);
  const bool c1 = d1 <= C.KAPPA * (fabsf(in.k) + fabsf(out.k)) + in.tol + out.tol + C.KAPPA0;
  const bool c2 = d2 <= C.KAPPA * (fabsf(br.k) + fabsf(fu.k)) + br.tol + fu.tol + C.KAPPA0;
  const bool c3 = fabsf(fu.k) <= C.KMAX + fu.tol;
  const bool c4 = rz3(C, A, Cc, E);
  score = d1 + d2;
  kfull = fu.k;
  return c1 && c2 && c3 && c4;
}

// The first condition of t5_select: the inner (a, b, c) and outer (c, d, e) curvatures agree.
__device__ __forceinline__ bool t5_in_out_agree(const MethodConst& C, const Circle3& in, const Circle3& out) {
  const float d1 = fabsf(in.k - out.k);
  return d1 <= C.KAPPA * (fabsf(in.k) + fabsf(out.k)) + in.tol + out.tol + C.KAPPA0;
}

// The conditions of t5_select after the first, in its order, stopping at the first failure:
// with t5_in_out_agree, the decision of t5_select without the score.
__device__ __forceinline__ bool t5_accept_rest(const MethodConst& C, const PointTol& A, const PointTol& B,
                                               const PointTol& Cc, const PointTol& D, const PointTol& E) {
  const Circle3 br = circle3(B, Cc, D);
  const Circle3 fu = circle3(A, Cc, E);
  const float d2 = fabsf(br.k - fu.k);
  if (!(d2 <= C.KAPPA * (fabsf(br.k) + fabsf(fu.k)) + br.tol + fu.tol + C.KAPPA0)) return false;
  if (!(fabsf(fu.k) <= C.KMAX + fu.tol)) return false;
  return rz3(C, A, Cc, E);
}

// Pseudo-angle of (x, y) in [0, 4): 0 along +x, 1 along +y, 2 along -x, 3 along -y,
// increasing with the azimuth inside each quadrant, from divisions only (the same binary32
// value on every device); the origin maps to 0.  Hits of a sensor are ordered by it, and
// |d psi / d phi| <= 1, so an azimuth window of half-width w is inside psi +- w.
__host__ __device__ __forceinline__ float pseudo_angle(float x, float y) {
  if (y >= 0.0f) {
    if (x >= 0.0f) {
      const float den = x + y;
      return den > 0.0f ? y / den : 0.0f;
    }
    return 1.0f + (-x) / (y - x);
  }
  if (x < 0.0f) return 2.0f + (-y) / (-x - y);
  return 3.0f + x / (x - y);
}

// ---- learned T5 selection ----
// The paper's selections include machine-learning methods (Sec. 1); here a small network
// can take the place of the two curvature-agreement conditions of a T5 while the radius
// and (a, c, e) r-z conditions stay.  Inputs (all but f5 are x / (x + y) of non-negative
// terms, in [0, 1)):
//   f0 = d1 / (d1 + rhs1)   f1 = d2 / (d2 + rhs2)   (differences against the cut tolerances)
//   f2 = d1 / (d1 + |kin| + |kout| + kappa0)   f3 = d2 / (d2 + |kbr| + |kfu| + kappa0)
//   f4 = (tol_in + tol_out) / ((tol_in + tol_out) + |kin| + |kout| + kappa0)
//   f5 = |kfu| / kmax
//   f6, f7 = residual / (residual + tolerance) of the r-z straightness of (a, c, e), (b, c, d)
// Network: h1 = relu(b1 + W1 f), h2 = relu(b2 + W2 h1), z = b3 + w3 . h2, every sum taken
// from the bias in index order; the candidate passes when z > 0.  The weights travel as a
// kernel parameter (by value, so a captured graph carries them) and each block stages them
// in shared memory, W2 transposed, where every read is a broadcast.
constexpr int T5_NF = 8, T5_NH = 16;
constexpr int T5_W1 = 0, T5_B1 = T5_W1 + T5_NH * T5_NF, T5_W2 = T5_B1 + T5_NH, T5_B2 = T5_W2 + T5_NH * T5_NH,
              T5_W3 = T5_B2 + T5_NH, T5_B3 = T5_W3 + T5_NH, T5_NPARAM = T5_B3 + 1;
constexpr int T5_SMEM_FLOATS = (T5_NPARAM + 3) & ~3;  // staged copy, float4-aligned sections
struct T5Mlp {
  float w[T5_NPARAM];
};

// Copies the weights into shared memory Ws (T5_SMEM_FLOATS, 16-byte aligned) with W2
// transposed (Ws[T5_W2 + j * T5_NH + k] = W2[k][j]); the caller synchronises the block.
__device__ __forceinline__ void t5_mlp_stage(const T5Mlp& M, float* Ws) {
  for (int i = threadIdx.x; i < T5_NPARAM; i += blockDim.x) {
    int d = i;
    if (i >= T5_W2 && i < T5_B2) {
      const int k = (i - T5_W2) / T5_NH, j = (i - T5_W2) % T5_NH;
      d = T5_W2 + j * T5_NH + k;
    }
    Ws[d] = M.w[i];
  }
}

__device__ __forceinline__ float frac_of(float x, float y) {
  const float den = x + y;
  return den > 0.0f ? x / den : 0.0f;
}

// The network on staged weights.  The loop runs over the first layer's units j; unit j's
// output is added, as term j, into all second-layer sums at once, so each sum still runs
// from its bias through j = 0, 1, ... in order, and the loop body stays short.
__device__ __forceinline__ float t5_mlp_logit(const float* Ws, const float (&f)[T5_NF]) {
  float a2[T5_NH];
#pragma unroll
  for (int k = 0; k < T5_NH; k++) a2[k] = Ws[T5_B2 + k];
#pragma unroll 1
  for (int j = 0; j < T5_NH; j++) {
    const float4 wa = *reinterpret_cast<const float4*>(Ws + T5_W1 + j * T5_NF);
    const float4 wb = *reinterpret_cast<const float4*>(Ws + T5_W1 + j * T5_NF + 4);
    float a = Ws[T5_B1 + j];
    a = a + wa.x * f[0];
    a = a + wa.y * f[1];
    a = a + wa.z * f[2];
    a = a + wa.w * f[3];
    a = a + wb.x * f[4];
    a = a + wb.y * f[5];
    a = a + wb.z * f[6];
    a = a + wb.w * f[7];
    const float h = a > 0.0f ? a : 0.0f;
    const float4* w2 = reinterpret_cast<const float4*>(Ws + T5_W2 + j * T5_NH);
#pragma unroll
    for (int q = 0; q < T5_NH / 4; q++) {
      const float4 v = w2[q];
      a2[4 * q] = a2[4 * q] + v.x * h;
      a2[4 * q + 1] = a2[4 * q + 1] + v.y * h;
      a2[4 * q + 2] = a2[4 * q + 2] + v.z * h;
      a2[4 * q + 3] = a2[4 * q + 3] + v.w * h;
    }
  }
  float z = Ws[T5_B3];
#pragma unroll
  for (int k = 0; k < T5_NH; k++) z = z + Ws[T5_W3 + k] * (a2[k] > 0.0f ? a2[k] : 0.0f);
  return z;
}

// The radius and (a, c, e) r-z conditions of a T5 candidate and, when both pass, the
// network's inputs f; score and curvature as in t5_select.
__device__ __forceinline__ bool t5_mlp_inputs(const MethodConst& C, const PointTol& A, const PointTol& B,
                                              const PointTol& Cc, const PointTol& D, const PointTol& E,
                                              float (&f)[T5_NF], float& score, float& kfull) {
  const Circle3 in = circle3(A, B, Cc);
  const Circle3 out = circle3(Cc, D, E);
  const Circle3 br = circle3(B, Cc, D);
  const Circle3 fu = circle3(A, Cc, E);
  const float d1 = fabsf(in.k - out.k);
  const float d2 = fabsf(br.k - fu.k);
  score = d1 + d2;
  kfull = fu.k;
  if (!(fabsf(fu.k) <= C.KMAX + fu.tol)) return false;
  float l, t;
  rz3_terms(C, A, Cc, E, l, t);
  if (!(l <= t)) return false;
  const float rhs1 = C.KAPPA * (fabsf(in.k) + fabsf(out.k)) + in.tol + out.tol + C.KAPPA0;
  const float rhs2 = C.KAPPA * (fabsf(br.k) + fabsf(fu.k)) + br.tol + fu.tol + C.KAPPA0;
  f[0] = frac_of(d1, rhs1);
  f[1] = frac_of(d2, rhs2);
  f[2] = frac_of(d1, fabsf(in.k) + fabsf(out.k) + C.KAPPA0);
  f[3] = frac_of(d2, fabsf(br.k) + fabsf(fu.k) + C.KAPPA0);
  f[4] = frac_of(in.tol + out.tol, fabsf(in.k) + fabsf(out.k) + C.KAPPA0);
  f[5] = fabsf(fu.k) / C.KMAX;
  f[6] = frac_of(l, t);
  rz3_terms(C, B, Cc, D, l, t);
  f[7] = frac_of(l, t);
  return true;
}

// t5_select with the network in place of the two curvature-agreement conditions (the
// score and curvature are the same); the network runs only when the radius and r-z
// conditions pass.
__device__ __forceinline__ bool t5_select_mlp(const MethodConst& C, const float* Ws, const PointTol& A,
                                              const PointTol& B, const PointTol& Cc, const PointTol& D,
                                              const PointTol& E, float& score, float& kfull) {
  float f[T5_NF];
  if (!t5_mlp_inputs(C, A, B, Cc, D, E, f, score, kfull)) return false;
  return t5_mlp_logit(Ws, f) > 0.0f;
}

// Score and full-circle curvature of a T5 whose decision is already known.
__device__ __forceinline__ void t5_measure(const PointTol& A, const PointTol& B, const PointTol& Cc,
                                           const PointTol& D, const PointTol& E, float& score, float& kfull) {
  const Circle3 in = circle3(A, B, Cc);
  const Circle3 out = circle3(Cc, D, E);
  const Circle3 br = circle3(B, Cc, D);
  const Circle3 fu = circle3(A, Cc, E);
  score = fabsf(in.k - out.k) + fabsf(br.k - fu.k);
  kfull = fu.k;
}

// ---- pLS helix ----
struct PlsHelix {
  float x0, y0, z0, R, cx, cy, cot, q, pt;
};

// Arc length of a chord on a circle of radius R: 2 R asin(chord / 2R), asin from two
// half-angle reductions and its Taylor series to the ninth power.
__device__ __forceinline__ float arc_length(float chord, float R) {
  float x = chord / (2.0f * R);
  if (x > 1.0f) x = 1.0f;
  const float x1 = x / sqrtf(2.0f * (1.0f + sqrtf(1.0f - x * x)));
  const float x2 = x1 / sqrtf(2.0f * (1.0f + sqrtf(1.0f - x1 * x1)));
  const float t = x2 * x2;
  const float as = x2 * (1.0f + t * (0.16666667f + t * (0.075f + t * (0.044642857f + t * 0.030381944f))));
  return 8.0f * R * as;
}

// sin and cos of a in [0, pi]: Taylor series at a / 4, then two angle doublings.
__device__ __forceinline__ void sin_cos_series(float a, float& s_out, float& c_out) {
  const float h = 0.25f * a;
  const float h2 = h * h;
  const float s = h * (1.0f - h2 / 6.0f * (1.0f - h2 / 20.0f * (1.0f - h2 / 42.0f * (1.0f - h2 / 72.0f * (1.0f - h2 / 110.0f)))));
  const float c = 1.0f - h2 / 2.0f * (1.0f - h2 / 12.0f * (1.0f - h2 / 30.0f * (1.0f - h2 / 56.0f * (1.0f - h2 / 90.0f * (1.0f - h2 / 132.0f)))));
  const float s2 = 2.0f * s * c;
  const float c2 = c * c - s * s;
  s_out = 2.0f * s2 * c2;
  c_out = c2 * c2 - s2 * s2;
}

// One anchor against the pLS helix: r-phi and r-z residuals inside windows that grow with
// the arc length from the reference point.  Adds the normalised squared residuals to score.
__device__ __forceinline__ bool pls_anchor(const MethodConst& C, const PlsHelix& h, const PointTol& X, float& score) {
  const float ddx = X.p.x - h.x0, ddy = X.p.y - h.y0;
  const float chord = sqrtf(ddx * ddx + ddy * ddy);
  const float s = arc_length(chord, h.R);
  const float ex = X.p.x - h.cx, ey = X.p.y - h.cy;
  const float dphi = sqrtf(ex * ex + ey * ey) - h.R;
  const float wphi = C.W0 + 0.003f * s + 0.015f * s * s / h.R + X.t.y;
  const float ez = X.p.z - (h.z0 + s * h.cot);
  const float wz = 0.05f + 0.002f * s + X.t.x + X.t.y * fabsf(h.cot);
  const float a = dphi / wphi, b = ez / wz;
  score = score + (a * a + b * b);
  return (fabsf(dphi) <= wphi) && (fabsf(ez) <= wz);
}

}  // namespace lst

namespace lst {

// Same decision as pls_anchor without the score.  The r-phi window grows with the arc
// length s from the reference point, and s <= (pi / 2) chord for any arc up to half a turn,
// so a residual beyond the window at s = 1.6 chord can never pass: that case is rejected
// before the arc-length series is evaluated.  Exact: the bound only removes candidates
// the full test rejects too.
// A cheap filter ahead of pls_anchor_accept: its first test (the r-phi residual against the
// window at s = 1.6 chord) with the square roots by rsqrtf (at most 2 ulp off) and the
// division by h.R as a product with inv_r = 1 / h.R; the window is widened by 1e-3 cm plus
// 2e-6 of the lengths involved, more than those errors and the roundings can move either
// side, so it keeps every anchor that test keeps.  Its survivors still go through
// pls_anchor_accept, which alone decides.
__device__ __forceinline__ bool pls_anchor_maybe_fast(const MethodConst& C, const PlsHelix& h, float inv_r,
                                                      const PointTol& X) {
  const float ddx = X.p.x - h.x0, ddy = X.p.y - h.y0;
  const float c2 = ddx * ddx + ddy * ddy;
  const float chord = c2 > 0.0f ? c2 * rsqrtf(c2) : 0.0f;
  const float ex = X.p.x - h.cx, ey = X.p.y - h.cy;
  const float e2 = ex * ex + ey * ey;
  const float dist = e2 > 0.0f ? e2 * rsqrtf(e2) : 0.0f;
  const float dphi = dist - h.R;
  const float smax = 1.6f * chord;
  const float wmax = (C.W0 + 0.003f * smax + 0.015f * smax * smax * inv_r + X.t.y) * 1.001f;
  return !(fabsf(dphi) > wmax + 1.0e-3f + 2.0e-6f * (dist + h.R + chord));
}

__device__ __forceinline__ bool pls_anchor_accept(const MethodConst& C, const PlsHelix& h, const PointTol& X) {
  const float ddx = X.p.x - h.x0, ddy = X.p.y - h.y0;
  const float chord = sqrtf(ddx * ddx + ddy * ddy);
  const float ex = X.p.x - h.cx, ey = X.p.y - h.cy;
  const float dphi = sqrtf(ex * ex + ey * ey) - h.R;
  const float smax = 1.6f * chord;
  const float wmax = (C.W0 + 0.003f * smax + 0.015f * smax * smax / h.R + X.t.y) * 1.001f;
  if (fabsf(dphi) > wmax) return false;
  const float s = arc_length(chord, h.R);
  const float wphi = C.W0 + 0.003f * s + 0.015f * s * s / h.R + X.t.y;
  if (!(fabsf(dphi) <= wphi)) return false;
  const float ez = X.p.z - (h.z0 + s * h.cot);
  const float wz = 0.05f + 0.002f * s + X.t.x + X.t.y * fabsf(h.cot);
  return fabsf(ez) <= wz;
}

}  // namespace lst
