"""The oracle's pins catch plausible mistakes.

Each case plants one mistake -- a dropped term, a wrong sign, a transposed operand, a wrong index
or constant -- in a copy of the oracle's C sources, builds that copy, and runs the oracle's pin
tests against it (PIC_ORACLE_LIB points the wrapper at the copy).  The case passes when a pin
fails.  Nothing here touches the GPU or the oracle the other tests use.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS_MAIN = ["tests/test_oracle_pins_numerics.py", "tests/test_oracle_pins_physics.py"]
PINS_ADJ = ["tests/test_oracle_pins_adjoint.py"]
PINS_SHEATH = ["tests/test_oracle_pins_sheath.py"]

# (name, file, text as written, text with the mistake, pin files expected to catch it)
MUTATIONS = [
    ("philox multiplier", "pic_oracle.c", "(uint64_t)0xD2511F53u * (uint64_t)c0",
     "(uint64_t)0xD2511F55u * (uint64_t)c0", PINS_MAIN),
    ("Thomas boundary sign", "pic_oracle.c", "if (j == 1) d += V_L;", "if (j == 1) d -= V_L;", PINS_MAIN),
    ("Thomas elimination sign", "pic_oracle.c", "dp[j] = (d - (-1.0) * dp[j - 1]) / den;",
     "dp[j] = (d + (-1.0) * dp[j - 1]) / den;", PINS_MAIN),
    ("wall Gauss term sign", "pic_oracle.c", "E[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / 2.0;",
     "E[0] = (phi[0] - phi[1]) / dx + rho[0] * dx / 2.0;", PINS_MAIN),
    ("Boris cross product transposed", "pic_oracle.c", "vm[0] + (vm[1] * t[2] - vm[2] * t[1])",
     "vm[0] + (vm[2] * t[1] - vm[1] * t[2])", PINS_MAIN),
    ("Boris second half kick dropped", "pic_oracle.c", "v[0] = vq[0] + h * E[0];", "v[0] = vq[0];",
     PINS_MAIN),
    ("null-collision probability linearised", "pic_oracle.c",
     "p_null[s] = (float)(1.0 - exp(-(double)nu_max[s] * c->dt));",
     "p_null[s] = (float)((double)nu_max[s] * c->dt);", PINS_MAIN),
    ("CIC deposit weights swapped", "pic_oracle.c", "R[c] += Wl;\n      R[c + 1] += Wr;",
     "R[c] += Wr;\n      R[c + 1] += Wl;", PINS_MAIN),
    ("wall half-cell volume dropped", "pic_oracle.c",
     "double vol = (j == 0 || j == N) ? 0.5 * s->dx : s->dx;", "double vol = s->dx;", PINS_MAIN),
    ("gather weights swapped", "pic_oracle.c", "Ex = (1.0 - f) * E[cc] + f * E[cc + 1];",
     "Ex = f * E[cc] + (1.0 - f) * E[cc + 1];", PINS_MAIN),
    ("elastic angle term dropped", "pic_oracle.c", "sqrt(1.0 - 2.0 * m / c->m_gas * (1.0 - cchi))",
     "sqrt(1.0 - 2.0 * m / c->m_gas)", PINS_MAIN),
    ("excitation loss dropped", "pic_oracle.c", "double sp2 = sqrt(2.0 * (En - c->E_ex) / m);",
     "double sp2 = sqrt(2.0 * En / m);", PINS_MAIN),
    ("ionization threshold dropped", "pic_oracle.c", "double Er = En - c->E_iz;", "double Er = En;",
     PINS_MAIN),
    ("charge exchange without a new velocity", "pic_oracle.c",
     "    v[0] = vt * n0;\n    v[1] = vt * n1;\n    v[2] = vt * n2;\n    tc->coll[3]++;",
     "    tc->coll[3]++;", PINS_MAIN),
    ("exponential load not truncated", "pic_oracle.c",
     "x = -lam * log(1.0 - u01(w[0]) * (1.0 - exp(-(double)N / lam)));",
     "x = -lam * log(1.0 - u01(w[0]));", PINS_MAIN),
    ("adjoint: gather position term dropped", "pic_adjoint.c",
     "lx[p] += ebar * (En[k0 + 1] - En[k0]);", "(void)En;", PINS_ADJ),
    ("adjoint: rotation not transposed", "pic_adjoint.c",
     "Lt[k] = m.M[s][0][k] * L[0] + m.M[s][1][k] * L[1] + m.M[s][2][k] * L[2];",
     "Lt[k] = m.M[s][k][0] * L[0] + m.M[s][k][1] * L[1] + m.M[s][k][2] * L[2];", PINS_ADJ),
    ("adjoint: flux share slope sign", "pic_adjoint.c", "(d > 0.0 ? -1.0 : (d < 0.0 ? 1.0 : 0.0))",
     "(d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0))", PINS_ADJ),
    ("adjoint: field transpose wall sign", "pic_adjoint.c", "if (k == 1) a -= mu[0] / dx;",
     "if (k == 1) a += mu[0] / dx;", PINS_ADJ),
    ("adjoint: initial field's bias term dropped", "pic_adjoint.c",
     "  for (int32_t j = 0; j <= N; ++j) gV += mu[j] / ((double)N * m.dx);\n  double gT",
     "  double gT", PINS_ADJ),
    ("adjoint: temperature chain factor", "pic_adjoint.c", "grad[1] = gT / (2.0 * c->T[0]);",
     "grad[1] = gT / c->T[0];", PINS_ADJ),
    ("adjoint: position update without 1/dx", "pic_adjoint.c", "lv[3 * p] += lx[p] * c->dt / m.dx;",
     "lv[3 * p] += lx[p] * c->dt;", PINS_ADJ),
    ("smoothing: wall node weights", "pic_oracle.c", "rho[0] = (old[0] + old[1]) / 2.0;",
     "rho[0] = (3.0 * old[0] + old[1]) / 4.0;", PINS_SHEATH),
    ("smoothing: interior weights", "pic_oracle.c",
     "rho[j] = (old[j - 1] + 2.0 * old[j] + old[j + 1]) / 4.0;",
     "rho[j] = (old[j - 1] + old[j] + old[j + 1]) / 3.0;", PINS_SHEATH),
    ("smoothing left out of the solve", "pic_oracle.c", "orc_smooth(N, s->cfg.smooth_passes, s->rho);",
     "(void)0;", PINS_SHEATH),
    ("recycled neutral leaves outward", "pic_oracle.c", "out->v[0] = side == 0 ? vx : -vx;",
     "out->v[0] = side == 0 ? -vx : vx;", PINS_SHEATH),
    ("recycled neutral not flux-weighted", "pic_oracle.c",
     "double vx = vt * sqrt(-2.0 * log(1.0 - u01(w[1])));",
     "double vx = vt * fabs(sqrt(-2.0 * log(1.0 - u01(w[1]))) * cos(2.0 * ORC_PI * u01(w[2])));",
     PINS_SHEATH),
    ("recycled neutral born a cell inside the right wall", "pic_oracle.c",
     "(double)s->N - 1.0 / 16777216.0", "(double)s->N - 1.0", PINS_SHEATH),
    ("recycling probability inverted", "pic_oracle.c", "if (!(u01(w[0]) < c->recycle)) return 0;",
     "if (!(u01(w[0]) >= c->recycle)) return 0;", PINS_SHEATH),
    ("neutral move without 1/dx", "pic_oracle.c", "double xh = p->x[i] + p->vx[i] * c->dt / s->dx;",
     "double xh = p->x[i] + p->vx[i] * c->dt;", PINS_SHEATH),
    ("neutral ionization without dt", "pic_oracle.c", "double P = 1.0 - exp(-c->K_iz * ne * c->dt);",
     "double P = 1.0 - exp(-c->K_iz * ne);", PINS_SHEATH),
    ("electron density without the half-cell wall volume", "pic_oracle.c",
     "s->ne[j] = s->w[0] * ((double)s->R[0][j] / TWO32) / vol;",
     "s->ne[j] = s->w[0] * ((double)s->R[0][j] / TWO32) / s->dx;", PINS_SHEATH),
    ("ionized neutral kept", "pic_oracle.c", "cnt[t][2]++;\n        keep[i] = 0;",
     "cnt[t][2]++;\n        keep[i] = 1;", PINS_SHEATH),
    ("ion of an ionized neutral takes the new electron's velocity", "pic_oracle.c",
     "plist_add(&nz_born[1][t], xh, v, p->id[i])", "plist_add(&nz_born[1][t], xh, e_new.v, p->id[i])",
     PINS_SHEATH),
    ("new electron at the ion mass", "pic_oracle.c", "double vt = sqrt(c->T_sec / c->mass[0]);",
     "double vt = sqrt(c->T_sec / c->mass[1]);", PINS_SHEATH),
    ("initial neutrals at the ion temperature", "pic_oracle.c",
     "const double vt = sqrt(c->T_rec / c->mass[1]);\n    uint32_t w[4];",
     "const double vt = sqrt(c->T[1] / c->mass[1]);\n    uint32_t w[4];", PINS_SHEATH),
    ("snapshot restore drops the ionization count", "pic_oracle.c", "get(&q, &s->nt_ionized, 8);",
     "q += 8;", PINS_SHEATH),
    ("countdown: the cap's expiry taken as a candidate", "pic_oracle.c",
     "if (fl >= (double)NEXT_KMAX) return NEXT_KMAX;", "if (fl >= (double)NEXT_KMAX) return NEXT_KMAX | NEXT_CAND;",
     PINS_MAIN),
    ("countdown: one step too long", "pic_oracle.c", "return ((uint32_t)fl + 1u) | NEXT_CAND;",
     "return ((uint32_t)fl + 2u) | NEXT_CAND;", PINS_MAIN),
    ("countdown: geometric parameter linearised", "pic_oracle.c", "log(v) / log1p(-(double)p_null)",
     "log(v) / (-(double)p_null)", PINS_MAIN),
]


def _build_copy(tmp, fname, old, new):
    src = os.path.join(tmp, "src")
    shutil.copytree(ORACLE, src, ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.py"))
    path = os.path.join(src, fname)
    text = open(path).read()
    assert text.count(old) == 1, f"the text to change occurs {text.count(old)} times in {fname}"
    open(path, "w").write(text.replace(old, new))
    lib = os.path.join(tmp, "liboracle_mut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-fopenmp", "-shared",
                    os.path.join(src, "pic_oracle.c"), os.path.join(src, "pic_adjoint.c"), "-o", lib, "-lm"],
                   check=True)
    return lib


@pytest.mark.parametrize("name,fname,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, fname, old, new, pins):
    lib = _build_copy(str(tmp_path), fname, old, new)
    env = dict(os.environ, PIC_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    # exit 1: a test failed (the mistake was caught); 0: every pin passed with the mistake in place
    assert r.returncode == 1, f"no pin caught '{name}' (pytest exit {r.returncode}):\n{r.stdout[-2000:]}"
