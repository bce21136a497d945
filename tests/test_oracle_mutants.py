"""Strength of the oracle's pins: planted mistakes must fail them.

Each mutant below is the oracle with one plausible mistake planted in a copy
of its source: a dropped term, a flipped sign, a transposed operand, a wrong
index or bound, a wrong root.  The copy is compiled on the CPU and the
oracle's pin tests run against it in a child process (PMP_ORACLE_LIB), with
-x; a mutant passes this test only if some pin fails.  The oracle itself is
never edited.  What each pin checks comes from the paper and the mathematics
(closed forms, conservation, Fig. 1, brute force), so a mutant that survived
would show a part of the oracle that only agrees with itself.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pmp_oracle.c")
DUAL = os.path.join(ROOT, "oracle", "dual.py")
# The last file checks the one-by-one evaluation that gives the expected
# values of the full-size GPU tests against the whole cycle.
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_create.py", "tests/test_oracle_extra.py",
        "tests/test_oracle_mass.py", "tests/test_oracle_batch.py", "tests/test_oracle_repro.py",
        "tests/test_oracle_one_by_one.py"]

# (name, the original text, its mutated form); the original occurs once.
# Equivalent mutants are left out: e.g. folding ghosts of a non-periodic axis
# too changes nothing, because the kernel is cut at that face and those
# ghosts only ever hold zeros; and the accretion limiter's eta needs no cap at
# 1 on a buffer from the sink deposit, where every pair removes at least
# rho - rho_Tr, so the summed removal is never below rho - rho_Tr (rounding
# is monotone) and the limited removal never exceeds it.
MUTANTS = [
    ("accretion removes instead of adding to the buffer's density row",
     "    dU[0] = -a;\n    for (int k = 0; k < 3; k++) dU[1 + k] = -(a * (U[1 + k] * inv));",
     "    dU[0] = a;\n    for (int k = 0; k < 3; k++) dU[1 + k] = -(a * (U[1 + k] * inv));"),
    ("internal energy without the kinetic term",
     "double eint = U[4] - ke2 * (0.5 * inv);",
     "double eint = U[4];"),
    ("gamma (gamma - 1) written gamma - 1",
     "double gg = P->gamma * (P->gamma - 1.0);",
     "double gg = P->gamma - 1.0;"),
    ("centre offset transposed (x_s - x_c)",
     "static double centre_offset(int c, double x) { return ((double)c + 0.5) - x; }",
     "static double centre_offset(int c, double x) { return x - ((double)c + 0.5); }"),
    ("V_snr sums cells instead of covered fractions",
     "        sw = sw + w;\n",
     "        sw = sw + 1.0;\n"),
    ("Bondi-Hoyle rate without lambda",
     "sqrt(lam2 * cinf2 + vinf2)",
     "sqrt(cinf2 + vinf2)"),
    ("accretion limiter without the 25% cap",
     "double al = a < P->cap * rho ? a : P->cap * rho;",
     "double al = a;"),
    ("Step 4 adds the removed mass to the sink with the wrong sign",
     "    acc[0] = acc[0] - b;",
     "    acc[0] = acc[0] + b;"),
    ("ghost fold takes face images only",
     "                            if (ox == 0 && oy == 0 && oz == 0) continue;\n"
     "                            if ((ox && !B->periodic[0])",
     "                            if ((ox != 0) + (oy != 0) + (oz != 0) != 1) continue;\n"
     "                            if ((ox && !B->periodic[0])"),
    ("momentum limiter takes the smaller root",
     "    return hi < 1.0 ? hi : 1.0;",
     "    if (lo > 0.0 && lo < 1.0) return lo;\n    return hi < 1.0 ? hi : 1.0;"),
    ("ejecta kinetic energy dropped",
     "G[FB_E * stride] = (Esn + Ekin) / Vsnr;",
     "G[FB_E * stride] = Esn / Vsnr;"),
    ("omega sub-points at the cell corner, not the mid-points",
     "double sx = ((double)ci + ((double)a + 0.5) / (double)S) - x;",
     "double sx = ((double)ci + ((double)a) / (double)S) - x;"),
    ("kernel membership with <= instead of <",
     "static int inside(double d2, double r2) { return d2 < r2; }",
     "static int inside(double d2, double r2) { return d2 <= r2; }"),
    ("momentum smoothing with rho instead of rho + q",
     "    double rn = U[0] + q;",
     "    double rn = U[0];"),
    ("Truelove term with the sign of rho - rho_Tr flipped",
     "    double tr = U[0] - rtr;\n    double a = bh >= tr ? bh : tr;\n    double inv",
     "    double tr = rtr - U[0];\n    double a = bh >= tr ? bh : tr;\n    double inv"),
    ("accretion energy row scaled by p_x instead of E",
     "    dU[4] = -(a * (U[4] * inv));",
     "    dU[4] = -(a * (U[1] * inv));"),
    ("radial momentum scaled by |d| instead of divided",
     "double s = c->d2 > 0.0 ? (w * Pv) / dist : 0.0;",
     "double s = c->d2 > 0.0 ? (w * Pv) * dist : 0.0;"),
    ("MC regime threshold compared with the wrong bound",
     "else if (RM <= P->RM_st)",
     "else if (RM <= P->RM_ej * 2.0)"),
    ("density floor dropped from the accretion limiter",
     "    double f = rho - P->rho_min;\n    al = al < f ? al : f;",
     "    double f = rho;\n    al = al < f ? al : f;"),
    ("sink gather mean density over one cell too many",
     "    double rho_inf = srho / (double)nk;",
     "    double rho_inf = srho / (double)(nk + 1);"),
    ("exp with one Taylor term fewer",
     "    double p = c[13];\n    for (int j = 12; j >= 0; j--) p = p * r + c[j];",
     "    double p = c[12];\n    for (int j = 11; j >= 0; j--) p = p * r + c[j];"),
    ("log without the low part of e ln2",
     "return ed * LN2_HI - ((hf - (s * (hf + R) + ed * LN2_LO)) - f);",
     "return ed * LN2_HI - ((hf - (s * (hf + R))) - f);"),
    ("App. A.1 rounding without the margin M",
     "        nbit = ceil_log2 + 52 + M;",
     "        nbit = ceil_log2 + 52;"),
    ("sink creation with a non-strict local maximum",
     "                            if (!(U[0] > rho2)) ok = 0;          /* (b) */",
     "                            if (!(U[0] >= rho2)) ok = 0;          /* (b) */"),
    ("sink creation ignoring the retained accretion buffer",
     "                if (!all_zero(D)) continue;                       /* (c) */",
     "                (void)D;"),
    ("particle-mesh deposit without omega",
     "    for (int f = 0; f < NF; f++) dU[f] = w * G[(MS_Q + f) * stride];",
     "    for (int f = 0; f < NF; f++) dU[f] = G[(MS_Q + f) * stride];"),
    ("v_COM adds gas momentum without the cell volume",
     "vc[a] = (sp[a] * V + pe[a]) / Msnr;",
     "vc[a] = (sp[a] + pe[a]) / Msnr;"),
    ("M_sf with the exponent's sign flipped",
     "double Msf = P->A_sf * or_pow(nH, -0.26);",
     "double Msf = P->A_sf * or_pow(nH, 0.26);"),
    ("P_snr with the exponent of M_sf",
     "prad = P->A_p * or_pow(nH, -0.17);",
     "prad = P->A_p * or_pow(nH, -0.26);"),
    ("ST radial momentum without the factor 2",
     "prad = sqrt(((2.0 * m) * P->eps_K) * Esn);",
     "prad = sqrt((m * P->eps_K) * Esn);"),
    ("accretion over the step without dt",
     "double K = ((mdot * P->dt) / V) / sumw;",
     "double K = (mdot / V) / sumw;"),
    ("r_acc clamped at half a cell instead of a quarter",
     "    if (racc < 0.25) racc = 0.25;",
     "    if (racc < 0.5) racc = 0.5;"),
    ("Step-4 momentum returned with the wrong sign",
     "    for (int k = 0; k < 3; k++) acc[1 + k] = fma(-b, U[1 + k] * inv, acc[1 + k]);",
     "    for (int k = 0; k < 3; k++) acc[1 + k] = fma(b, U[1 + k] * inv, acc[1 + k]);"),
    ("Step 4 without the cell's eta",
     "            double eta = sink_eta(P, S->dx, U, D);\n            return_add(eta, U, dU, acc);\n        }\n"
     "        p->m[s] = p->m[s] - acc[0] * V;",
     "            double eta = sink_eta(P, S->dx, U, D);\n            return_add(1.0, U, dU, acc);\n        }\n"
     "        p->m[s] = p->m[s] - acc[0] * V;"),
    ("App. A.1 ceil(log2 r) off by one at powers of two",
     "        int ceil_log2 = (m == 0.5) ? k - 1 : k;",
     "        int ceil_log2 = k;"),
    ("Eq. lambda's thermal term without the rho'/rho factor",
     "    double therm = (eint0 * rho1) / U[0];\n    double lhs",
     "    double therm = eint0;\n    double lhs"),
    ("Eq. lambda's constant term with rho' instead of 2 rho'",
     "    double C = p2 - (2.0 * rho1) * (E1 - therm);",
     "    double C = p2 - rho1 * (E1 - therm);"),
    ("particle-mesh V_K without the cell volume",
     "    double VK = sw * cell_volume(S->dx);",
     "    double VK = sw;"),
    ("omega sub-points of the y axis at the cell corner",
     "double sy = ((double)cj + ((double)b + 0.5) / (double)S) - y;",
     "double sy = ((double)cj + ((double)b) / (double)S) - y;"),
    ("sink relative velocity without the sink's own velocity",
     "    for (int a = 0; a < 3; a++) u[a] = sp[a] / srho - ps[a] / ms;",
     "    for (int a = 0; a < 3; a++) u[a] = sp[a] / srho;"),
    ("c_inf weighted by volume instead of mass",
     "        src = src + U[0] * cs;",
     "        src = src + cs;"),
    ("periodic wrap with C's remainder (negative for low ghosts)",
     "    int r = i % n;\n    return r < 0 ? r + n : r;",
     "    int r = i % n;\n    return r;"),
    ("kernel not cut at a non-periodic face",
     "                if (!S->periodic[0] && (ci < 0 || ci >= S->n[0])) continue;\n",
     ""),
    ("Step 4 without the cell volume",
     "        p->m[s] = p->m[s] - acc[0] * V;\n        p->px[s] = p->px[s] - acc[1] * V;\n"
     "        p->py[s] = p->py[s] - acc[2] * V;\n        p->pz[s] = p->pz[s] - acc[3] * V;\n    }\n    free(kc);",
     "        p->m[s] = p->m[s] - acc[0];\n        p->px[s] = p->px[s] - acc[1] * V;\n"
     "        p->py[s] = p->py[s] - acc[2] * V;\n        p->pz[s] = p->pz[s] - acc[3] * V;\n    }\n    free(kc);"),
    ("created sink mass without the cell volume",
     "                    double ms = (U[0] - rtr) * V;",
     "                    double ms = (U[0] - rtr);"),
    ("created sink's cell keeps its momentum instead of its velocity",
     "                    for (int a = 0; a < 3; a++) S->u[(int64_t)(1 + a) * S->fstride + c] = rtr * vel[a];",
     "                    (void)vel;"),
    ("auxiliary field updated without the limiter's eta",
     "X[(int64_t)f * stride + c] = x + eta * ((x / U[0]) * D[0]);",
     "X[(int64_t)f * stride + c] = x + ((x / U[0]) * D[0]);"),
    ("auxiliary field changed by its density, not its concentration",
     "X[(int64_t)f * stride + c] = x + eta * ((x / U[0]) * D[0]);",
     "X[(int64_t)f * stride + c] = x + eta * D[0];"),
    ("sink apply scales only the density row",
     "        double e = sink_eta(P, dx, U, D);\n        for (int f = 0; f < NF; f++) eta[f] = e;",
     "        double e = sink_eta(P, dx, U, D);\n        for (int f = 0; f < NF; f++) eta[f] = f == 0 ? e : 1.0;"),
    ("r_acc not clamped at r_K / 2",
     "    if (racc > 0.5 * P->r_K) racc = 0.5 * P->r_K;\n",
     ""),
    ("Step 4 reads eta at the unwrapped (ghost) cell instead of its owner",
     "            int64_t o = cell_index(B, kc[t].wi, kc[t].wj, kc[t].wk);\n            for (int f = 0; f < NF; f++) D[f] = B->u[(int64_t)f * B->fstride + o];\n            double eta = sink_eta(P, S->dx, U, D);\n            return_add(eta, U, dU, acc);\n        }\n        p->m[s]",
     "            int64_t o = cell_index(B, kc[t].ci, kc[t].cj, kc[t].ck);\n            for (int f = 0; f < NF; f++) D[f] = B->u[(int64_t)f * B->fstride + o];\n            double eta = sink_eta(P, S->dx, U, D);\n            return_add(eta, U, dU, acc);\n        }\n        p->m[s]"),
    ("Eq. mdot without rho_inf",
     "double mdot = (((4.0 * OR_PI) * rho_inf) * (r_bh * r_bh))",
     "double mdot = ((4.0 * OR_PI) * (r_bh * r_bh))"),
    ("App. A.1 error bound with half the machine epsilon",
     "if (ebuf) ebuf[o] = ebuf[o] + 2.220446049250313e-16 * fabs(B->u[o]);",
     "if (ebuf) ebuf[o] = ebuf[o] + 1.1102230246251565e-16 * fabs(B->u[o]);"),
    ("App. A.1 error bound from the added value instead of the sum",
     "if (ebuf) ebuf[o] = ebuf[o] + 2.220446049250313e-16 * fabs(B->u[o]);",
     "if (ebuf) ebuf[o] = ebuf[o] + 2.220446049250313e-16 * fabs(dU[f]);"),
    ("Eq. lambda's roots swapped when p . dp < 0",
     "        double Q = sq - B;\n        hi = Q / A;\n        lo = C / Q;",
     "        double Q = sq - B;\n        hi = C / Q;\n        lo = Q / A;"),
    ("Eq. lambda's roots swapped when p . dp >= 0",
     "        hi = Q != 0.0 ? C / Q : 0.0;\n        lo = Q / A;",
     "        hi = Q / A;\n        lo = Q != 0.0 ? C / Q : 0.0;"),
    ("accretion limiter caps at rho - rho_Tr instead of keeping it as a floor",
     "    al = al > t ? al : t;",
     "    al = al < t ? al : t;"),
    ("accretion limiter lets a negative limited removal through",
     "    if (al < 0.0) al = 0.0;\n    return al < a ? al / a : 1.0;",
     "    return al < a ? al / a : 1.0;"),
    ("Truelove density with J instead of J^2",
     "double ctr = ((P->J * P->J) * OR_PI) / (P->G * (dx * dx));",
     "double ctr = (P->J * OR_PI) / (P->G * (dx * dx));"),
    ("Truelove density without pi",
     "double ctr = ((P->J * P->J) * OR_PI) / (P->G * (dx * dx));",
     "double ctr = (P->J * P->J) / (P->G * (dx * dx));"),
    ("Truelove density over dx instead of dx^2",
     "double ctr = ((P->J * P->J) * OR_PI) / (P->G * (dx * dx));",
     "double ctr = ((P->J * P->J) * OR_PI) / (P->G * dx);"),
    ("stencil half-width truncated instead of rounded up",
     "static int stencil_halfwidth(double rK) { return (int)ceil(rK); }",
     "static int stencil_halfwidth(double rK) { return (int)rK; }"),
    ("r_acc in length units instead of cells",
     "    double racc = r_bh / S->dx;",
     "    double racc = r_bh;"),
    ("accretion kernel normalisation without the cell volume",
     "    double K = ((mdot * P->dt) / V) / sumw;",
     "    double K = (mdot * P->dt) / sumw;"),
    ("n_H without the mean mass per hydrogen",
     "    double nH = Msnr / (P->mu_H * Vsnr);",
     "    double nH = Msnr / Vsnr;"),
    ("ejecta density per SN mass instead of per volume",
     "    G[FB_Q * stride] = m / Vsnr;",
     "    G[FB_Q * stride] = m / Msnr;"),
    ("v_COM divided by the gas mass alone",
     "    for (int a = 0; a < 3; a++) vc[a] = (sp[a] * V + pe[a]) / Msnr;",
     "    for (int a = 0; a < 3; a++) vc[a] = (sp[a] * V + pe[a]) / Mgas;"),
    ("supernova energy row without the v_COM . p_rad term",
     "    dU[4] = fma(w, e, fma(vc[2], pr[2], fma(vc[1], pr[1], vc[0] * pr[0])));",
     "    dU[4] = w * e;"),
    ("radial direction not guarded at the particle's own cell centre",
     "    double s = c->d2 > 0.0 ? (w * Pv) / dist : 0.0;",
     "    double s = (w * Pv) / dist;"),
    ("accretion removal takes the smaller of K w and rho - rho_Tr",
     "    double a = bh >= tr ? bh : tr;",
     "    double a = bh <= tr ? bh : tr;"),
    ("omega over S^2 sub-points",
     "    return (double)cnt / (double)(S * S * S);",
     "    return (double)cnt / (double)(S * S);"),
    ("Eq. lambda's factor applied to the energy change too",
     "        eta[0] = 1.0; eta[1] = l; eta[2] = l; eta[3] = l; eta[4] = 1.0;",
     "        eta[0] = 1.0; eta[1] = l; eta[2] = l; eta[3] = l; eta[4] = l;"),
    ("Eq. lambda's factor applied to the density change too",
     "        eta[0] = 1.0; eta[1] = l; eta[2] = l; eta[3] = l; eta[4] = 1.0;",
     "        eta[0] = l; eta[1] = l; eta[2] = l; eta[3] = l; eta[4] = 1.0;"),
    ("ghost fold misses the outermost ghost layer",
     "                            if (gi < -g || gi >= nx + g || gj < -g || gj >= ny + g || gk < -g || gk >= nz + g) continue;",
     "                            if (gi <= -g || gi >= nx + g || gj <= -g || gj >= ny + g || gk <= -g || gk >= nz + g) continue;"),
    ("App. A.1 rounding drops one bit more than N_bit",
     "    if (nbit > 0) bits &= ~((((uint64_t)1) << nbit) - 1);",
     "    if (nbit > 0) bits &= ~((((uint64_t)1) << (nbit + 1)) - 1);"),
    ("created sink placed at the cell corner",
     "                    x[n] = (double)i + 0.5;",
     "                    x[n] = (double)i;"),
    ("sink creation's local maximum wraps across a non-periodic face",
     "                            if (a < 0 || a >= nx) { if (!S->periodic[0]) continue; a = (a + nx) % nx; }",
     "                            if (a < 0 || a >= nx) { a = (a + nx) % nx; }"),
    ("sink creation's local maximum includes cells exactly r_K away",
     "                            if (!(d2 < r2)) continue;\n                            int a = i + ox",
     "                            if (!(d2 <= r2)) continue;\n                            int a = i + ox"),
    ("created sink's cell keeps its energy density instead of its specific energy",
     "                    S->u[(int64_t)4 * S->fstride + c] = rtr * es;",
     "                    S->u[(int64_t)4 * S->fstride + c] = U[4];"),
    ("one-by-one evaluation misses the particles R cells below a cell",
     "        lo[a] = b[a] - R < 0 ? 0 : b[a] - R;",
     "        lo[a] = b[a] - R + 1 < 0 ? 0 : b[a] - R + 1;"),
    ("one-by-one fold adds the cell itself instead of its image",
     "                int st = deposit_at(P, S, p, bins, kc, gi, gj, gk, v, av);",
     "                int st = deposit_at(P, S, p, bins, kc, i, j, k, v, av);"),
    ("one-by-one state update without eta",
     "            out_new[NF * t + f] = zero ? U[f] : U[f] + eta[f] * D[f];",
     "            out_new[NF * t + f] = zero ? U[f] : U[f] + D[f];"),
    ("one-by-one Step 4 takes eta from the unfolded buffer",
     "            st = folded_at(P, S, p, bins, g, kc2, kc[q].wi, kc[q].wj, kc[q].wk, D, A);",
     "            st = deposit_at(P, S, p, bins, kc2, kc[q].wi, kc[q].wj, kc[q].wk, D, A);"),
    ("batched state ghost fill copies face ghosts only",
     "                    if (i >= 0 && i < M.n[0] && j >= 0 && j < M.n[1] && k >= 0 && k < M.n[2]) continue;",
     "                    if ((i < 0 || i >= M.n[0]) + (j < 0 || j >= M.n[1]) + (k < 0 || k >= M.n[2]) != 1) continue;"),
    ("batched Step 4 takes eta at a ghost image from the unfolded ghost",
     "            batch_fill_ghosts_n(T, owned, bcopy);\n",
     ""),
    ("batched limiter counts keep only the last patch's",
     "            tot[0] += c2[0];",
     "            tot[0] = c2[0];"),
    ("Eq. lambda keeps the whole momentum change when the quadratic has no real root",
     "    if (!(disc >= 0.0)) { *noroot = 1; return 0.0; }",
     "    if (!(disc >= 0.0)) { *noroot = 1; return 1.0; }"),
    ("Eq. lambda keeps the whole momentum change when both roots lie outside [0, 1]",
     "    if (hi < 0.0 || lo > 1.0) { *noroot = 1; return 0.0; }",
     "    if (hi < 0.0 || lo > 1.0) { *noroot = 1; return 1.0; }"),
    ("gathered gas mass without the cell volume",
     "    double Mgas = sr * V;",
     "    double Mgas = sr;"),
    ("batched fold reads the image from the patch on the wrong side",
     "int q = T->nb[26 * p + nb_slot(-ox, -oy, -oz)];",
     "int q = T->nb[26 * p + nb_slot(ox, oy, oz)];"),
    ("batched fold places a high-side image with the own patch's size",
     "gi[a] = cc[a] + (o[a] > 0 ? nq : 0) - (o[a] < 0 ? npa : 0);",
     "gi[a] = cc[a] + (o[a] > 0 ? npa : 0) - (o[a] < 0 ? npa : 0);"),
    ("batched fold skips images at corners and edges",
     "                                    if (ox == 0 && oy == 0 && oz == 0) continue;\n"
     "                                    int q = T->nb",
     "                                    if ((ox != 0) + (oy != 0) + (oz != 0) != 1) continue;\n"
     "                                    int q = T->nb"),
    ("batched owner maps a low-side ghost with its own patch's size",
     "w[a] = c[a] + (o[a] < 0 ? T->dims[3 * q + a] : 0) - (o[a] > 0 ? np_[a] : 0);",
     "w[a] = c[a] + (o[a] < 0 ? np_[a] : 0) - (o[a] > 0 ? np_[a] : 0);"),
]


def _compile(tmp, i, text):
    src = os.path.join(tmp, f"mutant_{i}.c")
    lib = os.path.join(tmp, f"libmutant_{i}.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fexcess-precision=standard", "-fPIC", "-shared", "-o", lib, src, "-lm"])
    return lib


def _pins_fail(lib):
    env = dict(os.environ, PMP_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, r.stdout[-400:]


def test_mutants_are_well_formed():
    src = open(SRC).read()
    names = set()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, f"{name}: the original text must occur once"
        assert old != new and name not in names
        names.add(name)


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    from concurrent.futures import ThreadPoolExecutor

    src = open(SRC).read()
    # control: the unchanged source, built and run the same way, passes
    failed, tail = _pins_fail(_compile(str(tmp_path), "control", src))
    assert not failed, tail

    def one(item):
        i, (name, old, new) = item
        failed, _ = _pins_fail(_compile(str(tmp_path), i, src.replace(old, new)))
        return name, failed

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(one, enumerate(MUTANTS)))
    survivors = [name for name, failed in results if not failed]
    assert not survivors, f"mistakes no pin catches: {survivors}"


# The forward-mode restatement behind the adjoint tests (oracle/dual.py),
# pinned by the C oracle's values and by central finite differences.
DUAL_MUTANTS = [
    ("quotient rule with the wrong sign",
     "(self.t * o.v - self.v * o.t) / (o.v * o.v)",
     "(self.t * o.v + self.v * o.t) / (o.v * o.v)"),
    ("product rule with a dropped term",
     "Dual(self.v * o.v, self.t * o.v + self.v * o.t)",
     "Dual(self.v * o.v, self.t * o.v)"),
    ("square-root derivative without the 2",
     "a.t / (2.0 * r) if r > 0 else 0.0",
     "a.t / r if r > 0 else 0.0"),
    ("power derivative without the exponent",
     "Dual(r, e * a.v ** (e - 1.0) * a.t)",
     "Dual(r, a.v ** (e - 1.0) * a.t)"),
    ("ST momentum without the ejecta energy's tangent",
     "prad = dsqrt(2.0 * m * params[\"eps_K\"] * E)",
     "prad = dsqrt(2.0 * m * params[\"eps_K\"] * E.v)"),
    ("tangent passed through cells where the limiter acts",
     "                if passmask[c]:\n                    tan[(f,) + c] += dU[f].t",
     "                tan[(f,) + c] += dU[f].t"),
    ("ejecta kinetic energy without the 1/2",
     "Ekin = (pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]) / (2.0 * m)",
     "Ekin = (pe[0] * pe[0] + pe[1] * pe[1] + pe[2] * pe[2]) / m"),
    ("power derivative with the exponent not lowered",
     "Dual(r, e * a.v ** (e - 1.0) * a.t)",
     "Dual(r, e * a.v ** e * a.t)"),
    ("cell offset tangent dropped (positions carry no derivative)",
     "d = [(float(cc) + 0.5) - xx for cc, xx in zip((i, j, k), xs)]",
     "d = [(float(cc) + 0.5) - Dual(xx.v) for cc, xx in zip((i, j, k), xs)]"),
]

_DUAL_RUNNER = (
    "import importlib.util, sys; sys.path.insert(0, {root!r});"
    "import oracle;"
    "spec = importlib.util.spec_from_file_location('oracle.dual', {path!r});"
    "m = importlib.util.module_from_spec(spec); sys.modules['oracle.dual'] = m;"
    "spec.loader.exec_module(m); oracle.dual = m;"
    "import pytest; sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', 'tests/test_oracle_dual.py']))"
)


def test_dual_mutants_are_well_formed():
    src = open(DUAL).read()
    for name, old, new in DUAL_MUTANTS:
        assert src.count(old) == 1, f"{name}: the original text must occur once"
        assert old != new


@pytest.mark.slow
def test_every_planted_mistake_in_the_dual_oracle_fails_a_pin(tmp_path):
    src = open(DUAL).read()

    def run(i, text):
        path = os.path.join(str(tmp_path), f"dual_mutant_{i}.py")
        with open(path, "w") as f:
            f.write(text)
        return subprocess.run([sys.executable, "-c", _DUAL_RUNNER.format(root=ROOT, path=path)], cwd=ROOT,
                              capture_output=True, text=True, timeout=600)

    control = run("control", src)  # the unchanged module through the same runner passes
    assert control.returncode == 0, control.stdout[-400:]
    survivors = []
    for i, (name, old, new) in enumerate(DUAL_MUTANTS):
        r = run(i, src.replace(old, new))
        if r.returncode == 0:
            survivors.append(name)
    assert not survivors, f"mistakes no pin catches: {survivors}"
