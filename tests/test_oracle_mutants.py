"""Planted mistakes in the oracle, each caught by the pin that names it (CPU only).

A pin is only worth what it catches. Each case below copies the oracle's C sources, plants one
plausible mistake by a textual replacement (the replaced text must occur exactly once), compiles
the copy with the oracle's flags and runs the named pins against it in a child process
(ORACLE_SO points the oracle wrapper at the copy). The pins must fail there, and the same pins
pass against the real oracle in the main suite. The in-tree oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

from oracle import build as obuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, replaced text, replacement, -k expression selecting the pins that must catch it)
MUTANTS = [
    ("fast speed from |B|^2 instead of B_n^2",
     "    double bn2 = w[5 + d] * w[5 + d] / w[0];\n", "    double bn2 = b2;\n",
     "P13_cfl_dt_uniform_state_cartesian or P13_riemann_dissipation"),
    ("phi width without sin(theta)",
     "    return ctr(o, 0, i) * sin(ctr(o, 1, j)) * w;\n", "    return ctr(o, 0, i) * w;\n",
     "P13_cfl_dt_spherical_widths"),
    ("theta width from the inner radial edge instead of the centre",
     "    if (d == 1) return ctr(o, 0, i) * w;\n", "    if (d == 1) return lo(o, 0, i) * w;\n",
     "P13_cfl_dt_spherical_widths"),
    ("CFL signal speed without |v_d|",
     "s += (fabs(w[1 + d]) + fast_speed(o, w, d)) / width(o, d, i, j, k);",
     "s += fast_speed(o, w, d) / width(o, d, i, j, k);",
     "P13_cfl_dt_uniform_state_cartesian"),
    ("TVDLF dissipation speed without |v_n|",
     "double c = fmax(fabs(wl[1 + d]) + cl, fabs(wr[1 + d]) + cr);", "double c = fmax(cl, cr);",
     "P13_riemann_dissipation"),
    ("pressure floor that does not rebuild the energy",
     "                    w[4] = o->p_floor;\n                    prim2cons(o, w, u);\n",
     "                    w[4] = o->p_floor;\n",
     "P14_floors"),
    ("density floor not counted",
     "if (u[RHO] < o->rho_floor) { u[RHO] = o->rho_floor; hits++; }",
     "if (u[RHO] < o->rho_floor) { u[RHO] = o->rho_floor; }",
     "P14_floors"),
    ("density floor that keeps the velocity instead of the momentum",
     "if (u[RHO] < o->rho_floor) { u[RHO] = o->rho_floor; hits++; }",
     "if (u[RHO] < o->rho_floor) { double f = o->rho_floor / u[RHO]; u[RHO] = o->rho_floor; "
     "u[M1] *= f; u[M2] *= f; u[M3] *= f; hits++; }",
     "P14_floors"),
    ("van Leer slope halved",
     "if (lim == LIM_VANLEER) return 2.0 * a * b / (a + b);",
     "if (lim == LIM_VANLEER) return a * b / (a + b);",
     "test_P4_linear_waves_second_order and 1-0-0"),
    ("energy flux without the -B_n (B.v) term",
     "    f[EN] = (u[EN] + ptot) * vn - bn * bv;\n", "    f[EN] = (u[EN] + ptot) * vn;\n",
     "test_P4_linear_waves_second_order and 2-0-0 or P3_brio_wu"),
    ("geometric hoop term of m_theta with the wrong sign",
     "+ cot * (rho * vp * vp - bp * bp)) / r;", "- cot * (rho * vp * vp - bp * bp)) / r;",
     "P1b"),
    ("Coriolis force without its factor 2",
     "F[c] = rho * cen[c] + 2.0 * rho * cor[c];", "F[c] = rho * cen[c] + rho * cor[c];",
     "P7"),
    ("work of gravity dropped from the energy",
     "                        Lc[EN] -= rho * vr * g;\n", "",
     "P5_P7_wind_residual_second_order"),
    ("Powell energy source with the wrong sign",
     "Lc[EN] -= db * (vr * br + vt * bt + vp * bp);", "Lc[EN] += db * (vr * br + vt * bt + vp * bp);",
     "P6b_powell"),
    ("Powell induction source from B instead of v",
     "Lc[B1] -= db * vr; Lc[B2] -= db * vt; Lc[B3] -= db * vp;", "Lc[B1] -= db * br; Lc[B2] -= db * bt; Lc[B3] -= db * bp;",
     "P6b_powell"),
    ("Linde term with the wrong sign",
     "Lc[B1] += gr[0]; Lc[B2] += gr[1]; Lc[B3] += gr[2];",
     "Lc[B1] -= gr[0]; Lc[B2] -= gr[1]; Lc[B3] -= gr[2];",
     "P6_linde"),
    ("map time weight measured from the later map",
     "    double ww = (tau - o->tm[m]) / (o->tm[m + 1] - o->tm[m]);\n",
     "    double ww = (o->tm[m + 1] - tau) / (o->tm[m + 1] - o->tm[m]);\n",
     "P8_boundary_time_interpolation"),
    ("probe longitude moved with the wrong sense of rotation",
     "double ph = lon - o->omega_si * tsi;", "double ph = lon + o->omega_si * tsi;",
     "P9_phi_wrap"),
    ("trilinear radial weights swapped",
     "double f = ((c & 1) ? wr : 1.0 - wr)", "double f = ((c & 1) ? 1.0 - wr : wr)",
     "P9_sampling_cell_centre"),
    ("probe v_phi left in the co-rotating frame",
     "q[4] = (acc[3] + o->omega * r * sin(th)) * O_V0;", "q[4] = acc[3] * O_V0;",
     "P9_probe_vphi"),
    ("CME cone test against sin instead of cos of the half-width",
     "double thr = cos(q[4]);", "double thr = sin(q[4]);",
     "P10_cme_footprint"),
    ("initial pressure falling as r^-gamma instead of r^-2 gamma",
     "w[4] = b[2] * pow(x, 2.0 * o->gamma);", "w[4] = b[2] * pow(x, o->gamma);",
     "IC_radial_expansion"),
    ("initial Parker spiral wound the wrong way",
     "w[7] = -w[5] * o->omega * r * sin(th) / w[1];", "w[7] = w[5] * o->omega * r * sin(th) / w[1];",
     "IC_radial_expansion"),
    ("driven face without the asymm flip of v_theta",
     "w[2] = -wm[2]; w[3] = -wm[3]; w[6] = -wm[6];", "w[2] = wm[2]; w[3] = -wm[3]; w[6] = -wm[6];",
     "P8_ghost_layers"),
    ("outer radius B_r continued as r^-1",
     "double f = (ctr(o, 0, src) / ctr(o, 0, gi)) * (ctr(o, 0, src) / ctr(o, 0, gi));",
     "double f = (ctr(o, 0, src) / ctr(o, 0, gi));",
     "P8_outer_radius"),
    ("tracer taken from the downwind side",
     "ft[s] = fr * (fr >= 0.0 ? cl : cr);", "ft[s] = fr * (fr >= 0.0 ? cr : cl);",
     "tracer_conserved or tracer_advection"),
    ("tracer clipped at zero only",
     "T[id] = fmin(fmax(T[id], 0.0), rho);", "T[id] = fmax(T[id], 0.0);",
     "tracer_clipped"),
    ("second SSP-RK2 stage without the average with U^n",
     "o->U[id] = 0.5 * o->U0[id] + 0.5 * (o->U1[id] + dt * o->L[id]);", "o->U[id] = o->U1[id] + dt * o->L[id];",
     "P3_sod_star_state or test_P4_linear_waves_second_order and 2-0-0"),
    ("cell volume with 1/2 instead of 1/3",
     "return (rp * rp * rp - rm * rm * rm) / 3.0 *", "return (rp * rp * rp - rm * rm * rm) / 2.0 *",
     "P5_steady_wind or P5_gravity_sign"),
    ("div B with the upper face's area on the lower face",
     "s += area(o, d, pl[0], pl[1], pl[2]) * 0.5 * (bc + bp) - area(o, d, i, j, k) * 0.5 * (bm + bc);",
     "s += area(o, d, pl[0], pl[1], pl[2]) * 0.5 * (bc + bp) - area(o, d, pl[0], pl[1], pl[2]) * 0.5 * (bm + bc);",
     "P6_divb"),
    ("Linde coefficient over the root of sum 1/dx^2",
     "double eta = o->divb_coef / (dt * sinv);", "double eta = o->divb_coef / (dt * sqrt(sinv));",
     "P6_linde"),
    ("GLM damping without c_h",
     "const double damp = exp(-o->glm_alpha * o->glm_ch * dt / o->glm_dmin);",
     "const double damp = exp(-o->glm_alpha * dt / o->glm_dmin);",
     "P12_glm_damping"),
    ("map times past the table clamped to the first map",
     "if (tau >= o->tm[n - 1]) { *m0 = *m1 = n - 1; *w = 0.0; return; }",
     "if (tau >= o->tm[n - 1]) { *m0 = *m1 = 0; *w = 0.0; return; }",
     "P8_boundary_time"),
    ("work of the rotating-frame force dropped from the energy",
     "Lc[EN] += vv[0] * F[0] + vv[1] * F[1] + vv[2] * F[2];", "Lc[EN] += 0.0;",
     "P5_P7_wind_residual"),
    ("HLL dissipation with the wrong sign",
     "f[v] = (sr * fl[v] - sl * fr[v] + sl * sr * (ur[v] - ul[v])) / (sr - sl);",
     "f[v] = (sr * fl[v] - sl * fr[v] - sl * sr * (ur[v] - ul[v])) / (sr - sl);",
     "P3_sod"),
    ("HLLD double-star energy with the wrong sign",
     "uss[EN] = us[s][EN] + (s ? 1.0 : -1.0) * sq * (vbs - vbss) * sg;",
     "uss[EN] = us[s][EN] - (s ? 1.0 : -1.0) * sq * (vbs - vbss) * sg;",
     "P3c"),
    ("HLLD double-star field weights swapped",
     "bss[c] = (sqL * bt[1][c] + sqR * bt[0][c]", "bss[c] = (sqL * bt[0][c] + sqR * bt[1][c]",
     "P3c or P3b"),
    ("band cells as wide inside the band as outside",
     "    else if (s <= sB) x = A + (s - sA) / f;\n", "    else if (s <= sB) x = A + (s - sA);\n",
     "P11_band_edges"),
    ("GLM psi star state with the wrong sign of the jump",
     "double ps = 0.5 * (pl + pr) - 0.5 * ch * (brr - bl);", "double ps = 0.5 * (pl + pr) + 0.5 * ch * (brr - bl);",
     "P12_glm_standing_wave"),
    ("GLM psi flux c_h instead of c_h^2",
     "o->FP[d][ib] = ch * ch * bs;", "o->FP[d][ib] = ch * bs;",
     "P12_glm_standing_wave"),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mutant_dir, name, old, new, pins):
    d = mutant_dir / name.replace(" ", "_").replace("/", "_").replace("|", "").replace("^", "")
    d.mkdir()
    srcs = []
    for s in obuild.SRCS:
        dst = d / os.path.basename(s)
        shutil.copyfile(s, dst)
        srcs.append(str(dst))
    main = d / "icarus_oracle.c"
    text = main.read_text()
    assert text.count(old) == 1, f"the text to replace occurs {text.count(old)} times"
    main.write_text(text.replace(old, new))
    so = obuild.compile_so(srcs, str(d / "liboracle_mutant.so"))
    env = dict(os.environ, ORACLE_SO=so, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-p", "no:cacheprovider", "-k", pins], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    tail = r.stdout[-2000:]
    assert r.returncode == 1 and " failed" in tail, f"pins [{pins}] did not catch it:\n{tail}"
