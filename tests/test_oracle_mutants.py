"""The oracle pins must catch plausible slips in the oracle.

Each case copies the oracle to a temporary directory, plants one mistake in
its C source (a transposed pose, a swapped u/v, a dropped gate, a wrong
rounding, ...), rebuilds it there and runs the pin suite against the planted
copy on the CPU.  The pin suite must fail for every mutant.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "pose_not_transposed": ("f->R[r * 3 + c] = Twd[c * 4 + r];", "f->R[r * 3 + c] = Twd[r * 4 + c];"),
    "translation_sign": ("f->t[i] = (float)(-s);", "f->t[i] = (float)(s);"),
    "u_v_swapped": ("*u = xh * rz;\n    *v = yh * rz;", "*v = xh * rz;\n    *u = yh * rz;"),
    "pixel_floor_not_round": ("float fu = floorf(u + 0.5f), fv = floorf(v + 0.5f);",
                              "float fu = floorf(u), fv = floorf(v);"),
    "sdf_sign": ("float sdf = d - P[2];", "float sdf = P[2] - d;"),
    "hidden_not_skipped": ("if (sdf < -p->mu) return 0;", ""),
    "no_truncation": ("float t = fminf(1.0f, sdf * fr->inv_mu);", "float t = sdf * fr->inv_mu;"),
    "plain_mean": ("*Fv = fmaf(*Fv, wf, t) / (wf + 1.0f);", "*Fv = (*Fv + t) * 0.5f;"),
    "weight_uncapped": ("*Wv = (uint8_t)(w + 1 < p->max_weight ? w + 1 : p->max_weight);",
                        "*Wv = (uint8_t)(w + 1);"),
    "depth_in_cm": ("float d = (float)D * 0.001f;\n    float sdf",
                    "float d = (float)D * 0.01f;\n    float sdf"),
    "no_sigma_gate": ("if (dist2 > fr->sigma2) return 0;", ""),
    "no_band_gate": ("if (!(fabsf(Ft) <= p->band)) return 0;", ""),
    "extrinsic_translation_flipped": ("rigid(fr->Rc, fr->tc, Pc[0], Pc[1], Pc[2], Ph);",
                                      "rigid(fr->Rc, fr->tc, Pc[0], Pc[1], Pc[2], Ph); Ph[0] -= 2 * fr->tc[0];"),
    "trilinear_axis_mixed": ("float c0 = lerpf(c00, c10, fr[1]);", "float c0 = lerpf(c00, c10, fr[0]);"),
    "colour_rounds_down": ("uint32_t nc = (cc * w + s[c] + ((w + 1u) >> 1)) / (w + 1u);",
                           "uint32_t nc = (cc * w + s[c]) / (w + 1u);"),
    "bilinear_weights_swapped": ("float top = fmaf(ax, p10 - p00, p00);", "float top = fmaf(ay, p10 - p00, p00);"),
    "colour_before_geometry": (
        "long long g = orc_geometry(p, &fr, F, W, depth);\n    long long c = orc_colour(p, &fr, F, W, C, depth, rgb);",
        "long long c = orc_colour(p, &fr, F, W, C, depth, rgb);\n    long long g = orc_geometry(p, &fr, F, W, depth);"),
    "normal_weight_sign": ("float dot = fmaf(n[0], Pc[0], fmaf(n[1], Pc[1], n[2] * Pc[2]));",
                           "float dot = -fmaf(n[0], Pc[0], fmaf(n[1], Pc[1], n[2] * Pc[2]));"),
    "eq10_additive": ("uint32_t wn = wp + (wq * (255u - wp) + 127u) / 255u;",
                      "uint32_t wn = wp + wq > 255u ? 255u : wp + wq;"),
    "no_08_gate": ("if (!(5u * wq > 4u * wp)) return 0;", ""),
    "unobserved_corner_used": ("if (corner(ctx, i0[0] + dx, i0[1] + dy, i0[2] + dz, &f) == 0) return 0;",
                               "corner(ctx, i0[0] + dx, i0[1] + dy, i0[2] + dz, &f);"),
}

# Slips in the ray caster (oracle/raycast.c), caught by tests/test_raycast_oracle.py.
RAYCAST_MUTANTS = {
    "rc_refine_wrong_end": ("float ts = fmaf(t - tp, Fp / (Fp - F), tp);", "float ts = fmaf(t - tp, F / (Fp - F), tp);"),
    "rc_normal_sign": ("if (good) n[a] = fp - fm;", "if (good) n[a] = fm - fp;"),
    "rc_back_faces": ("if (ok && has_prev && Fp > 0.0f && F <= 0.0f) {", "if (ok && has_prev && Fp * F <= 0.0f) {"),
    "rc_direction_not_normalised": ("c->R[3 * a + 2] * dc[2])) * nd;", "c->R[3 * a + 2] * dc[2]));"),
    "rc_colour_index_geometry_voxel": ("float q = floorf((vert[a] - v->origin[a]) * c->inv_sc);",
                                       "float q = floorf((vert[a] - v->origin[a]) * c->inv_sg);"),
    "rc_unobserved_used": ("if (v->W[idx] == 0) return 0;", ""),
    "rc_pose_transposed": ("d[a] = fmaf(c->R[3 * a], dc[0], fmaf(c->R[3 * a + 1], dc[1], c->R[3 * a + 2] * dc[2])) * nd;",
                           "d[a] = fmaf(c->R[a], dc[0], fmaf(c->R[a + 3], dc[1], c->R[a + 6] * dc[2])) * nd;"),
}
# Slips in mesh extraction and texture maps (oracle/mesh.c), caught by tests/test_mesh_oracle.py.
MESH_MUTANTS = {
    "mt_orientation_flipped": ("    if (dot < 0.0f) {\n        memcpy(out + 3", "    if (dot > 0.0f) {\n        memcpy(out + 3"),
    "mt_edge_from_wrong_end": ("out[ax] = fmaf(t, Pq - Pp, Pp);", "out[ax] = fmaf(t, Pp - Pq, Pq);"),
    "mt_inconsistent_split": ("static const int TET_AXES[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};",
                              "static const int TET_AXES[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 0, 1}};"),
    "mt_quad_wrong_diagonal": ("memcpy(tri, q[0], 12); memcpy(tri + 3, q[2], 12); memcpy(tri + 6, q[3], 12);",
                               "memcpy(tri, q[1], 12); memcpy(tri + 3, q[2], 12); memcpy(tri + 6, q[3], 12);"),
    "tx_green_blue_swapped": ("p[a] = fmaf((float)j, blue[a], fmaf((float)i, green[a], T[a]));",
                              "p[a] = fmaf((float)i, blue[a], fmaf((float)j, green[a], T[a]));"),
    "tx_divide_by_w": ("green[a] = (T[3 + a] - T[a]) / (float)(w - 1);", "green[a] = (T[3 + a] - T[a]) / (float)w;"),
    "tx_unobserved_colour_used": ("if ((c >> 24) == 0u) continue;", ""),
    "tx_size_truncated": ("float q = floorf(dist / size_pixel + 0.5f);", "float q = floorf(dist / size_pixel);"),
    "mc_face_order_reversed": ("{0, 4, 6, 2},  /* x = 0, normal -x */", "{0, 2, 6, 4},  /* x = 0, normal -x */"),
    "mc_fan_drops_last": ("for (int i = 1; i + 1 < m; ++i, ++n) {\n            memcpy(out + 9 * n, vert[s0], 12);",
                          "for (int i = 1; i + 2 < m; ++i, ++n) {\n            memcpy(out + 9 * n, vert[s0], 12);"),
    "mc_flat_triangles_allowed": ("flat = on_one_face(loop[s], loop[(s + i) % m], loop[(s + i + 1) % m]);", "flat = 0;"),
    "mc_runs_of_one_corner": ("while ((inside >> c[(j + 1) % 4]) & 1) j = (j + 1) % 4;", ""),
    "mc_inside_is_positive": ("if (Fc[k] < 0.0f) inside |= 1 << k;", "if (Fc[k] > 0.0f) inside |= 1 << k;"),
}
# Slips in the bilinear-cell decision of the photometric loss (oracle.c and the
# camera built in oracle/__init__.py), caught by tests/test_adjoint_oracle.py.
CELL_MUTANTS = {
    "cell_round_not_floor": ("oracle.c", "    *x0 = floorf(u);\n", "    *x0 = floorf(u + 0.5f);\n"),
    "cell_bound_w_minus_1": ("oracle.c", "*x0 + 1.0f <= (float)(W - 1) && *y0 >= 0.0f",
                             "*x0 <= (float)(W - 1) && *y0 >= 0.0f"),
    "cell_fx_cx_swapped": ("__init__.py", "Kr = np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1]], np.float32)",
                           "Kr = np.array([[cx, 0, fx], [0, fy, cy], [0, 0, 1]], np.float32)"),
    "cell_u_from_y": ("oracle.c", "    *x0 = floorf(u);\n    *y0 = floorf(v);", "    *x0 = floorf(v);\n    *y0 = floorf(u);"),
}
# Slips in camera tracking (oracle/icp.c), caught by tests/test_icp_oracle.py.
ICP_MUTANTS = {
    "icp_jacobian_n_cross_p": ("p[1] * nq[2] - p[2] * nq[1], p[2] * nq[0] - p[0] * nq[2],\n                                p[0] * nq[1] - p[1] * nq[0]",
                               "nq[1] * p[2] - nq[2] * p[1], nq[2] * p[0] - nq[0] * p[2],\n                                nq[0] * p[1] - nq[1] * p[0]"),
    "icp_solve_sign": ("double s = -g[i];", "double s = g[i];"),
    "icp_association_floor": ("const float fu = floorf(ux + 0.5f), fv = floorf(uy + 0.5f);",
                              "const float fu = floorf(ux), fv = floorf(uy);"),
    "icp_normal_away_from_camera": ("const float c[3] = {b[1] * a[2] - b[2] * a[1], b[2] * a[0] - b[0] * a[2], b[0] * a[1] - b[1] * a[0]};",
                                    "const float c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};"),
    "icp_pyramid_mixes_edges": ("if (fabsf(d - first) <= 0.03f) {", "if (fabsf(d - first) <= 3.0f) {"),
    "icp_level_centre": ("Kl[2] = (float)(((double)K[2] + 0.5) * s - 0.5);", "Kl[2] = (float)((double)K[2] * s);"),
    "icp_distance_gate_dropped": ("if (fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2])) > L->max_dist2) continue;", ""),
}
ALL = {**{k: ("oracle.c", "tests/test_oracle_pins.py") + v for k, v in MUTANTS.items()},
       **{k: ("icp.c", "tests/test_icp_oracle.py") + v for k, v in ICP_MUTANTS.items()},
       **{k: (v[0], "tests/test_adjoint_oracle.py") + v[1:] for k, v in CELL_MUTANTS.items()},
       **{k: ("raycast.c", "tests/test_raycast_oracle.py") + v for k, v in RAYCAST_MUTANTS.items()},
       **{k: ("mesh.c", "tests/test_mesh_oracle.py") + v for k, v in MESH_MUTANTS.items()}}


@pytest.mark.parametrize("name", sorted(ALL))
def test_pins_catch_mutant(tmp_path, name):
    fname, pins, before, after = ALL[name]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(before) == 1, "mutation site not found: " + name
    d = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    (d / "oracle" / fname).write_text(src.replace(before, after))
    shutil.copytree(os.path.join(ROOT, "tests"), d / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    os.symlink(os.path.join(ROOT, "paper_1602_06645_gb300"), d / "paper_1602_06645_gb300")
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d / "pytest.ini")
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-q", "-x",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=d, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
