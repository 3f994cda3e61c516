"""Planted mistakes in the oracle: each variant of oracle.cpp below carries one
plausible error (a flipped sign, a dropped term, a swapped index or operand,
an off-by-one in a rule) and must make at least one pin of
tests/test_oracle_pins.py fail. The variants are compiled on the CPU with the
oracle's own flags; the pins run against them in child processes
(TPC_ORACLE_LIB points the oracle package at the variant)."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (text in oracle.cpp, replacement)
MUTANTS = {
 'curvature_sign': ("R s2 = s - kap * dx;", "R s2 = s + kap * dx;"),
 'jac_ys_index': ("R Jys = dx * dTds;", "R Jys = dx * dTdq;"),
 'cov_transpose': ("acc = acc + Tm[i][l2] * J[j][l2];", "acc = acc + Tm[i][l2] * J[l2][j];"),
 'gain_swap': ("K1[i] = st.C[i][0] * in.W01 + st.C[i][1] * in.W11;", "K1[i] = st.C[i][0] * in.W11 + st.C[i][1] * in.W01;"),
 'w01_sign': ("in.W01 = -(S01 / det);", "in.W01 = (S01 / det);"),
 'basis_const': ("b[1] = ((R(3) * f3 - R(6) * f2) + R(4)) / R(6);", "b[1] = ((R(3) * f3 - R(6) * f2) + R(3)) / R(6);"),
 'dca_sign': ("R cy = y - cs / kap;", "R cy = y + cs / kap;"),
 'tape_div': ("return mk(q, a.id, 1.0 / b.v, b.id, -q / b.v);", "return mk(q, a.id, 1.0 / b.v, b.id, q / b.v);"),
 'tape_mul': ("return mk(a.v * b.v, a.id, b.v, b.id, a.v);", "return mk(a.v * b.v, a.id, a.v, b.id, b.v);"),
 'chord_not_arc': ("R l = d * A;", "R l = d;"),
 'z_uses_chord': ("st.p[1] = z + t * l;", "st.p[1] = z + t * d;"),
 't0_sign': ("W<R> zeta = a.vdrift * ((a.t - a.t0) - W<R>(that));", "W<R> zeta = a.vdrift * ((a.t + a.t0) - W<R>(that));"),
 'seedz_tf': ("double zeta = c.c.vdrift * ((c.cl.t[i] - c.c.t0) - c.c.tf_start);", "double zeta = c.c.vdrift * ((c.cl.t[i] - c.c.t0) + c.c.tf_start);"),
 'reject_count': ("reject = nacc >= c.p.min_acc_reject && in.chi2 > R(c.p.chi2_out);", "reject = nacc > c.p.min_acc_reject && in.chi2 > R(c.p.chi2_out);"),
 'no_inflate': ("st.C[i][j] = st.C[i][j] * R(c.p.refit_inflate);", "st.C[i][j] = st.C[i][j];"),
 'pass_dir': ("size_t i = (pass == 2) ? k : n - 1 - k;", "size_t i = (pass == 1) ? k : n - 1 - k;"),
 'nb_pred_sign': ("R py = yh - (yu - yh) * f;", "R py = yh + (yu - yh) * f;"),
 'chi2_drop_term': ("in.chi2 = in.r0 * (in.W00 * in.r0 + in.W01 * in.r1) + in.r1 * (in.W01 * in.r0 + in.W11 * in.r1);", "in.chi2 = in.r0 * (in.W00 * in.r0 + in.W01 * in.r1);"),
 'spline_vw_swap': ("R wb = bw[cc] * bv[bb];", "R wb = bw[bb] * bv[cc];"),
 'pick_z_weight': ("R d2 = (ry * ry) / vy + (rz * rz) / vz;", "R d2 = (ry * ry) / vy + (rz * rz) / vy;"),
 'no_inward_scale': ("st.C[i][j] = st.C[i][j] * R(c.p.inward_cov_scale);", "st.C[i][j] = st.C[i][j];"),
 'clean_one_sided': ("upc[h] = (up[h] >= 0 && dn[up[h]] == h) ? up[h] : -1;", "upc[h] = (up[h] >= 0) ? up[h] : -1;"),
 'start_two_hits': ("if (dnc[h] < 0 && upc[h] >= 0 && upc[upc[h]] >= 0) out[m++] = h;", "if (dnc[h] < 0 && upc[h] >= 0) out[m++] = h;"),
 'select_tie_high': ("(uint64_t)(0xFFFFFFFFu - (uint32_t)starts[k])", "(uint64_t)((uint32_t)starts[k])"),
 'select_gap_ge': ("if (kept < c.p.min_track_hits || maxgap > c.p.max_gap) continue;", "if (kept < c.p.min_track_hits || maxgap >= c.p.max_gap) continue;"),
 'seed_max_le': ("while (upc[cur] >= 0 && (int)H.size() < c.p.seed_max_hits) {", "while (upc[cur] >= 0 && (int)H.size() <= c.p.seed_max_hits) {"),
 'that_sign': ("that = c.c.tf_start - (sg * (double)zd) / c.c.vdrift;", "that = c.c.tf_start + (sg * (double)zd) / c.c.vdrift;"),
 'flag_scale_refit': ("if (flags & (1u << b)) e = e * R(sc[b]);", "if (flags & (1u << b)) e = e * R(sc[4 - b]);"),
 'nb_dmax_strict': ("if (!(D <= dmax)) continue;", "if (!(D < dmax)) continue;"),
 'rotation_curvature_term': ("J[2][0] = kap * sa;", "J[2][0] = -(kap * sa);"),
 'rotation_y_factor': ("J[0][0] = cf / c2;", "J[0][0] = c2 / cf;"),
 'cov_update_index': ("R v = st.C[i][j] - (K0[i] * HC0[j] + K1[i] * HC1[j]);", "R v = st.C[i][j] - (K0[i] * HC0[j] + K1[i] * HC0[j]);"),
 'merge_shift_sign': ("shift = (R)(sg * c.c.vdrift * (thi - thj));", "shift = (R)(sg * c.c.vdrift * (thj - thi));"),
 'merge_drop_cj': ("S[a][b] = st.C[a][b] + Cj[k];", "S[a][b] = st.C[a][b];"),
 'merge_rotation_dir': ("rotate<R>(c, st, sector_alpha(fj) - sector_alpha(fi))", "rotate<R>(c, st, sector_alpha(fi) - sector_alpha(fj))"),
 'merge_not_mutual': ("if (out[i] >= 0 && in[out[i]] == i) {", "if (out[i] >= 0) {"),
 'merge_row_rule': ("!(sg[j].rlo > sg[i].rhi)", "!(sg[j].rlo >= sg[i].rhi)"),
 'merge_frames': ("!(df == 0 || df == 1 || df == 17)", "!(df <= 2 || df >= 16)"),
 'merge_side': ("sg[j].ev != sg[i].ev || sg[j].side != sg[i].side) continue;", "sg[j].ev != sg[i].ev) continue;"),
 'merge_cholesky_sign': ("for (int k = 0; k < b; ++k) acc = acc - L[a][k] * L[b][k];", "for (int k = 0; k < b; ++k) acc = acc + L[a][k] * L[b][k];"),
 'refine_sign': ("double th = that - (sg * (double)val(z0)) / c.c.vdrift;", "double th = that + (sg * (double)val(z0)) / c.c.vdrift;"),
 'refine_side': ("double sg = c.cl.sector[idx[0]] < 18 ? 1.0 : -1.0;", "double sg = 1.0;"),
 'refine_upper': ("if (hi - th > T) th = th + ((hi - th) - T);", "if (hi - th > T) th = th - ((hi - th) - T);"),
 'refine_lower': ("if (lo - th < 0.0) th = th + (lo - th);", "if (lo - th < 0.0) th = th - (lo - th);"),
 'native_pad_centre_sign': ("float d = cl->y[i] - c->padc[r];", "float d = cl->y[i] + c->padc[r];"),
 'native_grad_no_pitch': ("double dyp = c.cl.pads ? (double)c.padw[c.cl.row[cluster_idx[a + q]]] : 1.0;", "double dyp = 1.0;"),
 'compress_update_measured': ("if (model) apply_update<float>(st, innovation<float>(st, dy, dz, sig2, sig2));", "if (model) apply_update<float>(st, innovation<float>(st, encode ? io.my[k] : dy, dz, sig2, sig2));"),
 'compress_floor': ("ry = (int32_t)std::nearbyint((io.my[k] - prey) * iqy);", "ry = (int32_t)std::floor((io.my[k] - prey) * iqy);"),
 'compress_step_axis': ("float dz = prez + (float)rz * qz;", "float dz = prez + (float)rz * qy;"),
 'field_cross_sign': ("d[3] = f * (w[4] * b0 - w[2] * b2);", "d[3] = f * (w[4] * b0 + w[2] * b2);"),
 'field_monomials': ("const R m[10] = {R(1), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};", "const R m[10] = {R(1), x, y, z, x * x, x * y, y * z, y * y, x * z, z * z};"),
 'field_pt_not_updated': ("out[4] = (q * cl) / rho;", "out[4] = q;"),
 'field_difference_sign': ("for (int k = 0; k < 5; ++k) st.p[k] = hx.p[k] + (full[k] - unif[k]);", "for (int k = 0; k < 5; ++k) st.p[k] = hx.p[k] - (full[k] - unif[k]);"),
 'field_not_rotated': ("b0 = B[0] * ca + B[1] * sa;\n      b1 = -(B[0] * sa) + B[1] * ca;", "b0 = B[0];\n      b1 = B[1];"),
 'zero_field_seed_unguarded': ("R q = kB_of<R>(c) != R(0) ? kap / kB_of<R>(c) : R(0);", "R q = kap / kB_of<R>(c);"),
 'merge_solve_operand': ("for (int k = 0; k < a; ++k) acc = acc - L[a][k] * w[k];", "for (int k = 0; k < a; ++k) acc = acc - L[a][k] * d[k];"),
 'joseph_no_kvk': ("      acc = acc + (K[i][0] * vy * K[j][0] + K[i][1] * vz * K[j][1]);\n", ""),
 'joseph_transposed': ("for (int l = 0; l < 5; ++l) acc = acc + AC[i][l] * A[j][l];", "for (int l = 0; l < 5; ++l) acc = acc + AC[i][l] * A[l][j];"),
 'margin_dcut_gradient': ("mg->take(std::fabs(Dv - (double)val(dmax)) / (2.0 * std::sqrt(Dv * kf) * xr));", "mg->take(std::fabs(Dv - (double)val(dmax)) / (2.0 * std::sqrt(Dv) * xr));"),
 'vertex_z_sign': ("Innov<R> in = innovation<R>(sv, R(0.0), R(zv), R(vvar), R(vvar));", "Innov<R> in = innovation<R>(sv, R(0.0), R(-zv), R(vvar), R(vvar));"),
 'vertex_no_chi2': ("      chi2 = chi2 + in.chi2;\n      ndf += 2;\n      st = sv;", "      ndf += 2;\n      st = sv;"),
 'margin_tie_skipped': ("      mg->take(g > 0.0 ? std::fabs(Dp - Db) / (g * xr) : 0.0);", "      mg->take(g > 0.0 && Dp != Db ? std::fabs(Dp - Db) / (g * xr) : INFINITY);"),
}


def _caught(src, name, tmp):
    a, b = MUTANTS[name]
    d = os.path.join(tmp, name)
    os.makedirs(d)
    with open(os.path.join(d, "oracle.cpp"), "w") as f:
        f.write(src.replace(a, b))
    lib = os.path.join(d, "liborc.so")
    subprocess.check_call(["g++", *oracle.CXXFLAGS, os.path.join(d, "oracle.cpp"), "-o", lib])
    env = dict(os.environ, TPC_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py",
                        "tests/test_parity_checker.py", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode != 0


def test_every_planted_mistake_fails_a_pin():
    with open(oracle.SRC) as f:
        src = f.read()
    for name, (a, _) in MUTANTS.items():
        assert src.count(a) == 1, f"{name}: the text to mutate is no longer unique in oracle.cpp"
    with tempfile.TemporaryDirectory() as tmp, \
            cf.ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2))) as ex:
        caught = dict(zip(MUTANTS, ex.map(lambda n: _caught(src, n, tmp), MUTANTS)))
    survivors = [n for n, c in caught.items() if not c]
    assert not survivors, f"planted mistakes not caught by any pin: {survivors}"
