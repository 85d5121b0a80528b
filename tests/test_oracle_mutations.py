"""Planted mistakes: every pin of the oracle together must catch each of them.

Each mutation below is one plausible slip in the oracle's source (a dropped term, a
flipped sign, a transposed operand, a wrong index or bound).  The test builds a copy of
lst_oracle.c with that one change (on the CPU, in a temporary directory), runs the oracle
pins (test_oracle_pins.py, test_oracle_cuts.py, test_oracle_enumeration.py,
test_oracle_tilted.py, test_oracle_endcap_2s.py, test_oracle_t5_mlp.py) against the
copy in a child process, and requires at least one of them to fail.  A mutation that no
pin catches would be a part of the oracle that nothing but the oracle itself vouches for.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lst_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_cuts.py", "tests/test_oracle_enumeration.py",
        "tests/test_oracle_tilted.py", "tests/test_oracle_endcap_2s.py", "tests/test_oracle_t5_mlp.py"]

# Two widening terms are left out on purpose: the endcap part of the bending slack
# (rho_a + rho_b) (|sin dphi| + 0.05) and the sensor gap in a barrel module's r_max.  No
# true track needs them (worst-case 3-sigma radial errors on 0.81-0.9 GeV endcap pairs pass
# the bending cut without the first; the second moves the 0.8 GeV edge by 0.2-0.4 %, inside
# the 0.03 cm r-phi slack), so no physics pin can tell them from their absence; the
# oracle-GPU identity fixes them.  Two more slips have no effect on any event tried
# (full PU200-like and high-occupancy events): dropping the neighbour module's half width
# from the connection map's phi window (the window's bending term is far wider than any
# accepted pair needs), dropping a tilted module's radial span from its connection-map box
# (the map's r-z corner bound stays permissive for every pair tried) and letting removed
# pT5s remove pT3s (no pT3 overlapping a removed
# pT5 in two MDs survives the other rules), so they are not listed either.
#
# (name, exact source text, replacement)
MUTATIONS = [
    # hit-pair bending (MD and LS)
    ("bend: sign of the cross component", "float U = a->x * dy - a->y * dx;", "float U = a->x * dy + a->y * dx;"),
    ("bend: sign in the radial component", "float V = a->x * dx + a->y * dy;", "float V = a->x * dx - a->y * dy;"),
    ("bend: radial tolerance dropped from W", "float W = V + rs * a->r;", "float W = V;"),
    ("bend: outward requirement dropped", "return (W > 0.0f) && (fabsf(U) <= W * T + E);",
     "return (fabsf(U) <= W * T + E);"),
    ("bend: inner module's slope for the LS", "if (!(pair_bend(a, b, TB) && pair_rz(a, b))) return 0;",
     "if (!(pair_bend(a, b, a->T) && pair_rz(a, b))) return 0;"),
    # hit-pair r-z
    ("rz: sign of the pointing term", "float f = a->z * b->r - a->r * b->z;", "float f = a->z * b->r + a->r * b->z;"),
    ("rz: z resolution dropped", "(a->zeta * b->r + b->zeta * a->r + a->rho * fabsf(b->z) + b->rho * fabsf(a->z))",
     "(a->rho * fabsf(b->z) + b->rho * fabsf(a->z))"),
    ("rz: radial resolution dropped", "(a->zeta * b->r + b->zeta * a->r + a->rho * fabsf(b->z) + b->rho * fabsf(a->z))",
     "(a->zeta * b->r + b->zeta * a->r)"),
    ("rz: luminous region from dz", "float tol = C_Z0MAX * dr +", "float tol = C_Z0MAX * dz +"),
    # MD direction against the chord (LS tail)
    ("md_dir: chord-angle term dropped", "float tol = clen * (dlen * clen * C_HINV + C_EDIR + (lo->rho + up->rho));",
     "float tol = clen * (C_EDIR + (lo->rho + up->rho));"),
    ("md_dir: direction error dropped", "float tol = clen * (dlen * clen * C_HINV + C_EDIR + (lo->rho + up->rho));",
     "float tol = clen * (dlen * clen * C_HINV + (lo->rho + up->rho));"),
    ("md_dir: cross product sign", "float crs = fabsf(dx * cy - dy * cx);\n  float tol = clen * (dlen * clen",
     "float crs = fabsf(dx * cy + dy * cx);\n  float tol = clen * (dlen * clen"),
    ("ls: outer MD direction not tested", "return md_dir(a, au, cx, cy, clen) && md_dir(b, bu, cx, cy, clen);",
     "return md_dir(a, au, cx, cy, clen);"),
    ("ls: inner MD direction not tested", "return md_dir(a, au, cx, cy, clen) && md_dir(b, bu, cx, cy, clen);",
     "return md_dir(b, bu, cx, cy, clen);"),
    # barrel exit
    ("exit: test dropped", "if (barrel_to_disk && !exit_ok(a, b, rnext_a, zb_half)) return 0;", ""),
    ("exit: start from the outer anchor", "float rexit = a->r + (b->r - a->r) * t;", "float rexit = b->r + (b->r - a->r) * t;"),
    ("exit: one side only", "float Zb = b->z > 0.0f ? zb_half : -zb_half;", "float Zb = zb_half;"),
    # T3
    ("rz3: operands transposed", "*lhs = fabsf(zqp * dps - zsp * dpq);", "*lhs = fabsf(zqp * dpq - zsp * dps);"),
    ("rz3: resolution terms dropped",
     "p->zeta * fabsf(dps - dpq) + q->zeta * dps + s->zeta * dpq +\n         (p->rho + s->rho) * fabsf(zqp) + (p->rho + q->rho) * fabsf(zsp);",
     "(p->rho + s->rho) * fabsf(zqp) + (p->rho + q->rho) * fabsf(zsp);"),
    ("mid_dir: arc difference as a sum", "(fabsf(dbc - dab) + 0.02f * clen)", "((dbc + dab) + 0.02f * clen)"),
    ("mid_dir: direction error dropped",
     "float tol = clen * (dlen * (fabsf(dbc - dab) + 0.02f * clen) * C_HINV + C_EDIR + (b->rho + bu->rho));",
     "float tol = clen * (dlen * (fabsf(dbc - dab) + 0.02f * clen) * C_HINV + (b->rho + bu->rho));"),
    ("t3 radius: comparison flipped", "return (slack <= 0.0f) || (prod >= C_K3 * slack);",
     "return (slack <= 0.0f) || (prod <= C_K3 * slack);"),
    ("t3: radius not tested", "  return t3_radius(a, b, c);\n}", "  return 1;\n}"),
    # curvature and T5
    ("curv3: factor 2 dropped", "*k = 2.0f * cross / prod;", "*k = cross / prod;"),
    ("curv3: sagitta tolerance not squared", "*tol = 8.0f * dmax / (dsp * dsp);", "*tol = 8.0f * dmax / dsp;"),
    ("t5: inner/outer difference as a sum", "c->d1 = fabsf(c->kin - c->kout);", "c->d1 = fabsf(c->kin + c->kout);"),
    ("t5: bridge triple index", "curv3(P[1], P[2], P[3], &c->kbr, &c->tbr, NULL, NULL, NULL);",
     "curv3(P[1], P[2], P[4], &c->kbr, &c->tbr, NULL, NULL, NULL);"),
    ("t5: radius from the inner triple", "int c3 = fabsf(c.kfu) <= C_KMAX + c.tfu;", "int c3 = fabsf(c.kin) <= C_KMAX + c.tfu;"),
    ("t5: r-z of the wrong triple", "int c4 = rz3(P[0], P[2], P[4]);", "int c4 = rz3(P[0], P[1], P[4]);"),
    ("t5: relative slack dropped", "c->rhs1 = C_KAPPA * (fabsf(c->kin) + fabsf(c->kout)) + c->tin + c->tout + C_KAPPA0;",
     "c->rhs1 = c->tin + c->tout + C_KAPPA0;"),
    ("t5: score without the bridge term", "*score = c.d1 + c.d2;", "*score = c.d1;"),
    # pLS helix, lookup, anchors
    ("pls: centre on the wrong side", "o->cx = s->x0 + qR * uy;", "o->cx = s->x0 - qR * uy;"),
    ("pls: cot from the radius", "o->cot = s->pz / o->pt;", "o->cot = s->pz / o->R;"),
    ("arc_len: one half-angle reduction lost", "return 8.0f * R * as;", "return 4.0f * R * as;"),
    ("sincos: doubling lost", "*s_out = 2.0f * s2 * c2;", "*s_out = s2 * c2;"),
    ("pls lookup: z neighbours dropped", "for (int dz = -1; dz <= 1; dz++) add_row_cands", "for (int dz = 0; dz <= 0; dz++) add_row_cands"),
    ("pls lookup: disks on the wrong side", "int side0 = p->cot > 0.0f ? 11 : 6;", "int side0 = p->cot > 0.0f ? 6 : 11;"),
    ("pls lookup: phi neighbours dropped", "for (int d = -1; d <= 1; d++) {\n    int kk", "for (int d = 0; d <= 0; d++) {\n    int kk"),
    ("pls anchor: curvature term dropped", "float wphi = C_W0 + 0.003f * s + 0.015f * s * s / p->R + X->rho;",
     "float wphi = C_W0 + 0.003f * s + X->rho;"),
    ("pls anchor: chord for arc length", "float ez = X->z - (p->z0 + s * p->cot);", "float ez = X->z - (p->z0 + chord * p->cot);"),
    ("pls anchor: r-z window ignored", "return (unsigned)(fabsf(dphi) <= wphi) | (unsigned)(fabsf(ez) <= wz) << 1;",
     "return (unsigned)(fabsf(dphi) <= wphi) | 2u;"),
    ("pt5: curvature window without 1/R", "return fabsf(fabsf(kf) - 1.0f / p->R) <= C_KPT5 / p->R + tf;",
     "return fabsf(fabsf(kf) - 1.0f / p->R) <= C_KPT5 + tf;"),
    # joins and bookkeeping
    ("md join: last upper hit skipped", "for (uint32_t j = bin_off[2 * m + 1]; j < bin_off[2 * m + 2]; j++) {",
     "for (uint32_t j = bin_off[2 * m + 1]; j + 1 < bin_off[2 * m + 2]; j++) {"),
    ("ls join: first MD of a module skipped", "for (uint32_t b = md_off[B]; b < md_off[B + 1]; b++) {",
     "for (uint32_t b = md_off[B] + 1; b < md_off[B + 1]; b++) {"),
    ("t3 join: inner MD as the shared one", "uint32_t b = ls.p[2 * l1 + 1];", "uint32_t b = ls.p[2 * l1];"),
    ("t5 join: continue from MD b", "for (uint32_t i2 = t3_off[c]; i2 < t3_off[c + 1]; i2++) {",
     "for (uint32_t i2 = t3_off[b]; i2 < t3_off[b + 1]; i2++) {"),
    ("map: wedge centres added", "double dc = remainder(cA - cB, 2 * M_PI);", "double dc = remainder(cA + cB, 2 * M_PI);"),
    ("map: r-z tolerance without the luminous region", "double rhs = 15.0 * drmax +", "double rhs = 1.5 * drmax +"),
    ("module constants: 2S z tolerance of a PS module", "*zeta = m->stype == 0 ? 0.15f : 1.30f;", "*zeta = 0.15f;"),
    ("hit radius includes z", "o->z = ev->z[h];\n  o->r = sqrtf(o->x * o->x + o->y * o->y);",
     "o->z = ev->z[h];\n  o->r = sqrtf(o->x * o->x + o->y * o->y + o->z * o->z);"),
    # tilted barrel modules
    ("tilted: bending slope without the section's radial span",
     "rmax = (double)m->surf + 0.5 * ((double)m->emax - (double)m->emin) * fabs(tan(t)) + (double)m->gap * cos(t);",
     "rmax = (double)m->surf + (double)m->gap * cos(t);"),
    ("tilted: radial tolerance dropped", "*rho = (float)(0.15 * fabs(sin((double)m->tilt)));", "*rho = 0.0f;"),
    ("tilted: z tolerance of a 2S strip", "*zeta = (float)(0.15 * fabs(cos((double)m->tilt)));", "*zeta = 1.30f;"),
    ("endcap 2S: radial tolerance of a PS ring", "*rho = m->stype == 0 ? 0.15f : 2.55f;", "*rho = 0.15f;"),
    # duplicate removal and candidates
    ("dedup: pT5 overlap threshold 2", "if (count_shared(pls_md5 + 5 * x, 5, pls_md5 + 5 * y, 5) >= 3 && better",
     "if (count_shared(pls_md5 + 5 * x, 5, pls_md5 + 5 * y, 5) >= 2 && better"),
    ("dedup: pT3 against pT5 overlap threshold 3",
     "if (out->alive_pt5[z] && count_shared(pls_md3 + 3 * x, 3, pls_md5 + 5 * z, 5) >= 2) dead = 1;",
     "if (out->alive_pt5[z] && count_shared(pls_md3 + 3 * x, 3, pls_md5 + 5 * z, 5) >= 3) dead = 1;"),
    ("dedup: T5 stage ignores pT3s", "if (out->alive_pt3[z] && count_shared(mx, 5, pls_md3 + 3 * z, 3) >= 3) dead = 1;", ""),
    ("dedup: tie broken the wrong way", "return sy < sx || (sy == sx && y < x);", "return sy < sx || (sy == sx && y > x);"),
    ("tc: pLS used by a pT3 stays a candidate", "out->pls_tc[p] = !(used5[p] || used3[p]);", "out->pls_tc[p] = !used5[p];"),
    ("tc: T5 pT without the field constant", "pt = C_KB / fabsf(t5k.p[x]);", "pt = 1.0f / fabsf(t5k.p[x]);"),
    ("tc: a triplet seed listed with four pixel hits", "(ev->pls[pls].n_hits == 3 ? 3 : 4)", "(4)"),
    # azimuth order of the hits inside a sensor
    ("hit order: second-quadrant pseudo-angle reversed", "return 1.0f + (-x) / (y - x);", "return 1.0f + y / (y - x);"),
    ("hit order: input order kept", "while (j > bin_off[s] && (psi[bin_list[j - 1]] > psi[h] ||",
     "while (j > bin_off[s] && 0 && (psi[bin_list[j - 1]] > psi[h] ||"),
    # learned T5 selection: its inputs, the network, where its decision goes
    ("t5 net: f0 against the bridge/full tolerance", "f[0] = frac_of(c->d1, c->rhs1);", "f[0] = frac_of(c->d1, c->rhs2);"),
    ("t5 net: f3 with the inner curvature", "f[3] = frac_of(c->d2, fabsf(c->kbr) + fabsf(c->kfu) + C_KAPPA0);",
     "f[3] = frac_of(c->d2, fabsf(c->kin) + fabsf(c->kfu) + C_KAPPA0);"),
    ("t5 net: f4 with the bridge error", "f[4] = frac_of(c->tin + c->tout,", "f[4] = frac_of(c->tbr + c->tout,"),
    ("t5 net: f5 times k_max", "f[5] = fabsf(c->kfu) / C_KMAX;", "f[5] = fabsf(c->kfu) * C_KMAX;"),
    ("t5 net: f6 on (a, b, e)", "rz3_terms(P[0], P[2], P[4], &l, &t);\n  f[6]", "rz3_terms(P[0], P[1], P[4], &l, &t);\n  f[6]"),
    ("t5 net: f7 on (a, c, d)", "rz3_terms(P[1], P[2], P[3], &l, &t);", "rz3_terms(P[0], P[2], P[3], &l, &t);"),
    ("t5 net: ratio inverted", "return den > 0.0f ? x / den : 0.0f;", "return den > 0.0f ? y / den : 0.0f;"),
    ("t5 net: first layer not rectified", "h1[j] = a > 0.0f ? a : 0.0f;", "h1[j] = a;"),
    ("t5 net: W1 transposed", "a = a + w1[j * ORA_T5_NF + i] * f[i];", "a = a + w1[i * ORA_T5_NH + j] * f[i];"),
    ("t5 net: W2 transposed", "a = a + w2[k * ORA_T5_NH + j] * h1[j];", "a = a + w2[j * ORA_T5_NH + k] * h1[j];"),
    ("t5 net: b2 read from b1", "float a = b2[k];", "float a = b1[k];"),
    ("t5 net: output bias dropped", "float z = b3[0];", "float z = 0.0f;"),
    ("t5 net: decision z >= 0", "c1 = c2 = t5_mlp_logit(mlp, f) > 0.0f;", "c1 = c2 = t5_mlp_logit(mlp, f) >= 0.0f;"),
    ("t5 net: replaces the radius condition", "c1 = c2 = t5_mlp_logit(mlp, f) > 0.0f;",
     "c1 = c3 = t5_mlp_logit(mlp, f) > 0.0f;"),
]


def _mutant(tmp, k, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {k}: source text not found exactly once"
    path = os.path.join(tmp, f"m{k}.c")
    open(path, "w").write(src.replace(old, new))
    lib = os.path.join(tmp, f"m{k}.so")
    subprocess.run(["gcc", "-O1", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-I", os.path.join(ROOT, "oracle"), "-o", lib, path, "-lm", "-lpthread"], check=True)
    env = dict(os.environ, LST_ORACLE_LIB=lib, PYTHONDONTWRITEBYTECODE="1")
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider", "-m",
                            "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
        return r.returncode, r.stdout[-600:]
    except subprocess.TimeoutExpired:
        return -1, "timeout"


@pytest.fixture(scope="module")
def outcomes():
    with tempfile.TemporaryDirectory() as tmp:
        n = max(2, min(16, os.cpu_count() or 2))
        with cf.ThreadPoolExecutor(n) as ex:
            futs = {name: ex.submit(_mutant, tmp, k, old, new) for k, (name, old, new) in enumerate(MUTATIONS)}
            return {name: f.result() for name, f in futs.items()}


def test_unmutated_oracle_passes_the_pins():
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, outcomes):
    rc, out = outcomes[name]
    assert rc not in (0, 5), f"no pin fails with the mistake planted ({name}):\n{out}"
