"""Planted mistakes: each entry below changes one line of the oracle the way a
plausible slip would (a dropped term, a wrong sign, index or bound, a
transposed operand, a reversed tie), compiles that copy into a private
library, and runs the pin module named beside it against it.  The module
must fail: a pin that passes a broken oracle pins nothing.

The copies are built in a temporary directory and loaded by the child
pytest through SFF_ORACLE_LIB; the oracle's own sources and library are not
touched."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORE, INTERP, SGM, SIFT = (os.path.join(ROOT, "oracle", f) for f in
                           ("sff_oracle.c", "sff_interp_oracle.c", "sff_sgm_oracle.c", "sff_sift_oracle.c"))
FEATURES, COST, MATCH, FILTER = ("tests/test_oracle_features.py", "tests/test_oracle_philox_cost.py",
                                 "tests/test_oracle_match.py", "tests/test_oracle_filter_seeds.py")

# (name, source file, text, replacement, pin module that must fail)
MUTATIONS = [
    # scale space and features (Sec. 3.1)
    ("smoothing rounds down", CORE, "(uint8_t)((sum + n * n / 2) / (n * n));", "(uint8_t)(sum / (n * n));", FEATURES),
    ("smoothing window shifted", CORE, "for (int j = -n / 2; j <= n / 2 - 1; j++)",
     "for (int j = -n / 2 + 1; j <= n / 2; j++)", FEATURES),
    ("patch offset off by one", CORE, "int xx = clampi(x + n * (j - 3), 0, w - 1);",
     "int xx = clampi(x + n * (j - 4), 0, w - 1);", FEATURES),
    ("quantisation truncates", CORE, "if (a % d != 0 && a < 0) q -= 1;", "if (0) q -= 1;", FEATURES),
    ("quantisation clamps at -127", CORE, "q = clampi(q, -128, 127);", "q = clampi(q, -127, 127);", FEATURES),
    ("norm wrong", CORE, "nn += q * q;", "nn += q * q + (q < 0);", FEATURES),
    # cost (Eq. 1) and the random numbers
    ("stereo position sign", CORE, "c += ssd(a, fat(V->ste, V->w, V->h, px - V->sigma * u[2], py));",
     "c += ssd(a, fat(V->ste, V->w, V->h, px + V->sigma * u[2], py));", COST),
    ("cross position uses d0", CORE, "c += ssd(a, fat(V->crs, V->w, V->h, px + u[0] - V->sigma * u[3], py + u[1]));",
     "c += ssd(a, fat(V->crs, V->w, V->h, px + u[0] - V->sigma * u[2], py + u[1]));", COST),
    ("Philox with nine rounds", CORE, "for (int r = 0; r < 10; r++) {", "for (int r = 0; r < 9; r++) {", COST),
    ("Philox Weyl constants swapped", CORE, "if (r > 0) { k[0] += W0; k[1] += W1; }",
     "if (r > 0) { k[0] += W1; k[1] += W0; }", COST),
    ("offset range 2n", CORE, "uint32_t j = (uint32_t)(((uint64_t)r * (uint64_t)(4 * n)) >> 32);",
     "uint32_t j = (uint32_t)(((uint64_t)r * (uint64_t)(2 * n)) >> 32);", COST),
    # initialisation, propagation, random search
    ("initial argmin keeps the last tie", CORE,
     "u[3] = (int16_t)(V->sigma * (tx - cx));\n                        int32_t c = cost_at(V, px, py, u);\n"
     "                        if (c < best_c) { best_c = c; memcpy(best_u, u, sizeof best_u); }",
     "u[3] = (int16_t)(V->sigma * (tx - cx));\n                        int32_t c = cost_at(V, px, py, u);\n"
     "                        if (c <= best_c) { best_c = c; memcpy(best_u, u, sizeof best_u); }", MATCH),
    ("strict epipolar sign", CORE, "if (V->sigma * (px - qx) >= 0)", "if (V->sigma * (px - qx) > 0)", MATCH),
    ("propagation takes ties", CORE,
     "if (c < best_c) { best_c = c; memcpy(best_u, snap_f + 4 * j, sizeof best_u); }",
     "if (c <= best_c) { best_c = c; memcpy(best_u, snap_f + 4 * j, sizeof best_u); }", MATCH),
    ("column-only colours", CORE, "if (((x / n + y / n) & 1) != colour) continue;",
     "if (((x / n) & 1) != colour) continue;", MATCH),
    ("successors instead of predecessors", CORE,
     "int qx[2] = {x - dx * n, x}, qy[2] = {y, y - dy * n};\n"
     "                        for (int k = 0; k < 2; k++) {\n"
     "                            if (qx[k] < 0 || qx[k] >= w || qy[k] < 0 || qy[k] >= h) continue;\n"
     "                            size_t j = (size_t)qy[k] * w + qx[k];\n"
     "                            if (snap_c[j]",
     "int qx[2] = {x + dx * n, x}, qy[2] = {y, y + dy * n};\n"
     "                        for (int k = 0; k < 2; k++) {\n"
     "                            if (qx[k] < 0 || qx[k] >= w || qy[k] < 0 || qy[k] >= h) continue;\n"
     "                            size_t j = (size_t)qy[k] * w + qx[k];\n"
     "                            if (snap_c[j]", MATCH),
    ("direction order", CORE, "static const int DIRS[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};",
     "static const int DIRS[4][2] = {{1, 1}, {1, -1}, {-1, -1}, {-1, 1}};", MATCH),
    ("counter without the iteration", CORE,
     "uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u}, r[4];",
     "uint32_t ctr[4] = {(uint32_t)i, 0u, (uint32_t)(s + 4 * mirror), 0u}, r[4];", MATCH),
    ("counter without the pass", CORE,
     "uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u}, r[4];",
     "uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)(s), 0u}, r[4];", MATCH),
    ("counter words swapped", CORE,
     "uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u}, r[4];",
     "uint32_t ctr[4] = {(uint32_t)it, (uint32_t)i, (uint32_t)(s + 4 * mirror), 0u}, r[4];", MATCH),
    ("key words swapped", CORE, "const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};",
     "const uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};", MATCH),
    ("random search takes ties", CORE,
     "                    int32_t c = cost_at(&V, x, y, cand);\n"
     "                    if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }\n"
     "                }\n        }",
     "                    int32_t c = cost_at(&V, x, y, cand);\n"
     "                    if (c <= cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }\n"
     "                }\n        }", MATCH),
    ("disparities not clamped", CORE,
     "                    if (cu[2] < 0) cu[2] = 0;\n                    if (cu[3] < 0) cu[3] = 0;\n"
     "                    int16_t cand[4] = {(int16_t)cu[0], (int16_t)cu[1], (int16_t)cu[2], (int16_t)cu[3]};\n"
     "                    int32_t c = cost_at(&V, x, y, cand);\n"
     "                    if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }\n"
     "                }\n        }",
     "                    int16_t cand[4] = {(int16_t)cu[0], (int16_t)cu[1], (int16_t)cu[2], (int16_t)cu[3]};\n"
     "                    int32_t c = cost_at(&V, x, y, cand);\n"
     "                    if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }\n"
     "                }\n        }", MATCH),
    # consistency, region filter, seeds
    ("tau_c exclusive", CORE, "keep[i] = mx <= prm->tau_c;", "keep[i] = mx < prm->tau_c;", FILTER),
    ("consistency error capped at 254", CORE, "cerr[i] = (uint8_t)(sum > 255 ? 255 : sum);",
     "cerr[i] = (uint8_t)(sum > 254 ? 254 : sum);", FILTER),
    ("s_c inclusive", CORE, "if (joinable && tail < prm->region_min)", "if (joinable && tail <= prm->region_min)",
     FILTER),
    ("diagonal neighbour", CORE, "static const int NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};",
     "static const int NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {1, 1}};", FILTER),
    ("any neighbour joinable", CORE, "} else if (rejected[j]) {", "} else {", FILTER),
    ("seed tie on cost reversed", CORE, "(cerr[i] == cerr[best] && fwd_cost[i] < fwd_cost[best]))",
     "(cerr[i] == cerr[best] && fwd_cost[i] > fwd_cost[best]))", FILTER),
    ("seed tie on cerr reversed", CORE, "if (best < 0 || cerr[i] < cerr[best] ||",
     "if (best < 0 || cerr[i] <= cerr[best] ||", FILTER),
    ("seed cerr not stored", CORE, "sd->cost = fwd_cost[best]; sd->cerr = cerr[best];",
     "sd->cost = fwd_cost[best]; sd->cerr = 0;", FILTER),
    ("partial edge blocks dropped", CORE,
     "for (int x = bx; x < bx + 3 && x < w; x++) {\n                    int i = y * w + x;\n"
     "                    if (!keep[i]) continue;",
     "for (int x = bx; x < bx + 3 && x < w && bx + 3 <= w; x++) {\n                    int i = y * w + x;\n"
     "                    if (!keep[i]) continue;", FILTER),
    # disparity fill (SGM)
    ("census window transposed", SGM, "for (int j = -3; j <= 3; j++)\n                for (int i = -4; i <= 4; i++) {",
     "for (int j = -4; j <= 4; j++)\n                for (int i = -3; i <= 3; i++) {", "tests/test_oracle_sgm.py"),
    ("census test not strict", SGM, "if (q < c) bits |= (uint64_t)1 << k;", "if (q <= c) bits |= (uint64_t)1 << k;",
     "tests/test_oracle_sgm.py"),
    ("grey weights", SGM, "(uint8_t)((p[0] + 2 * p[1] + p[2] + 2) >> 2);", "(uint8_t)((2 * p[0] + p[1] + p[2] + 2) >> 2);",
     "tests/test_oracle_sgm.py"),
    ("cost clamped at the wrong side", SGM, "const int xr = x - d < 0 ? 0 : x - d;",
     "const int xr = x + d >= W ? W - 1 : x + d;", "tests/test_oracle_sgm.py"),
    ("P1 and P2 swapped", SGM, "if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;",
     "if (d > 0 && prev[d - 1] + P2 < best) best = prev[d - 1] + P2;", "tests/test_oracle_sgm.py"),
    ("minimum not subtracted", SGM, "L[i + d] = (uint16_t)(C[i + d] + best - m);", "L[i + d] = (uint16_t)(C[i + d] + best);",
     "tests/test_oracle_sgm.py"),
    ("a direction dropped", SGM, "for (int r = 0; r < 8; r++) {\n        for (size_t i = 0; i < n; i++) S[i] += L[r][i];",
     "for (int r = 0; r < 7; r++) {\n        for (size_t i = 0; i < n; i++) S[i] += L[r][i];", "tests/test_oracle_sgm.py"),
    ("winner ties to the highest d", SGM, "if (S[p * D + d] < S[p * D + best]) best = d;",
     "if (S[p * D + d] <= S[p * D + best]) best = d;", "tests/test_oracle_sgm.py"),
    ("fill threshold exclusive", SGM, "if (e <= tau_c && (bg < 0 || e < bge", "if (e < tau_c && (bg < 0 || e < bge",
     "tests/test_oracle_sgm.py"),
    ("fill seed kind", SGM, "s.kind = 1;", "s.kind = 0;", "tests/test_oracle_sgm.py"),
    # SIFT-PCA cost
    ("cell index transposed", SIFT, "const int cell = (j / 3) * 4 + i / 3;", "const int cell = (i / 3) * 4 + j / 3;",
     "tests/test_oracle_sift.py"),
    ("clip at 0.25", SIFT, "if (v[k] > 0.2f) v[k] = 0.2f;", "if (v[k] > 0.25f) v[k] = 0.25f;",
     "tests/test_oracle_sift.py"),
    ("quantisation not rounded", SIFT, "const int qv = (int)(u * 512.0f + 0.5f);", "const int qv = (int)(u * 512.0f);",
     "tests/test_oracle_sift.py"),
    ("sample offset off by one", SIFT,
     "const int qx = clampi(x + (i - 6) * n, 0, w - 1), qy = clampi(y + (j - 6) * n, 0, h - 1);",
     "const int qx = clampi(x + (i - 5) * n, 0, w - 1), qy = clampi(y + (j - 6) * n, 0, h - 1);",
     "tests/test_oracle_sift.py"),
    ("bias sign", SIFT, "phi[p * 4 + c] = t - bias[c];", "phi[p * 4 + c] = t + bias[c];", "tests/test_oracle_sift.py"),
    ("axis sign convention", SIFT, "const double sg = v[big] < 0.0 ? -1.0 : 1.0;",
     "const double sg = v[big] < 0.0 ? 1.0 : -1.0;", "tests/test_oracle_sift.py"),
    ("cost window 5 x 5", SIFT, "    for (int j = -3; j <= 3; j++)\n        for (int i = -3; i <= 3; i++) {\n"
     "            const int x = px + i * n, y = py + j * n;",
     "    for (int j = -2; j <= 2; j++)\n        for (int i = -2; i <= 2; i++) {\n"
     "            const int x = px + i * n, y = py + j * n;", "tests/test_oracle_sift.py"),
    ("cost window at stride 1", SIFT, "const int x = px + i * n, y = py + j * n;", "const int x = px + i, y = py + j;",
     "tests/test_oracle_sift.py"),
    ("cost without the cross view", SIFT, "            c = c + dist3(a, r);\n", "", "tests/test_oracle_sift.py"),
    ("cost cross view shifted by d0", SIFT,
     "clampi(x + u[0] - sigma * u[3], 0, w - 1)) * 4;", "clampi(x + u[0] - sigma * u[2], 0, w - 1)) * 4;",
     "tests/test_oracle_sift.py"),
    ("squared distances", SIFT, "return sqrtf((dx * dx + dy * dy) + dz * dz);", "return (dx * dx + dy * dy) + dz * dz;",
     "tests/test_oracle_sift.py"),
    ("third component dropped", SIFT, "return sqrtf((dx * dx + dy * dy) + dz * dz);", "return sqrtf(dx * dx + dy * dy);",
     "tests/test_oracle_sift.py"),
    # dense interpolation
    ("Y from cx", INTERP, "X[1] = (y - P->cy) * Z / P->focal;", "X[1] = (y - P->cx) * Z / P->focal;",
     "tests/test_oracle_interp.py"),
    ("ridge on the constant term", INTERP, "        M[0] += lam;\n        M[4] += lam;",
     "        M[0] += lam;\n        M[4] += lam;\n        M[8] += lam;", "tests/test_oracle_interp.py"),
    ("no ridge towards A = I", INTERP, "            rhs[a * 4 + a] += lam;  /* towards A = I */", "            /* dropped */",
     "tests/test_oracle_interp.py"),
    ("weights from d^2", INTERP,
     "const double w = exp(-P->alpha * sqrt((double)nb[i].d2) / P->dist_unit);\n        const double r[3]",
     "const double w = exp(-P->alpha * ((double)nb[i].d2) / P->dist_unit);\n        const double r[3]",
     "tests/test_oracle_interp.py"),
    ("unweighted centroid", INTERP, "for (int j = 0; j < 3; j++) cen[j] += w * X0[j];\n        wsum += w;",
     "for (int j = 0; j < 3; j++) cen[j] += X0[j];\n        wsum += 1.0;", "tests/test_oracle_interp.py"),
    ("reprojection clamp at 2", INTERP, "triangulate(P, x, y, d0 > 1.0 ? d0 : 1.0, X0);",
     "triangulate(P, x, y, d0 > 2.0 ? d0 : 2.0, X0);", "tests/test_oracle_interp.py"),
    ("no reprojection clamp", INTERP, "triangulate(P, x, y, d0 > 1.0 ? d0 : 1.0, X0);", "triangulate(P, x, y, d0, X0);",
     "tests/test_oracle_interp.py"),
    ("no test of Z1", INTERP, "if (!(X1[2] > 0.0)) {", "if (0) {", "tests/test_oracle_interp.py"),
    ("closest seed ties to the upper index", INTERP, "if (best < 0 || d2 < bd) { best = i; bd = d2; }",
     "if (best < 0 || d2 <= bd) { best = i; bd = d2; }", "tests/test_oracle_interp.py"),
    ("d1 = 0 without motion", INTERP, "        out[3] = (float)d0;\n        return;\n    }\n    double X0[3]",
     "        out[3] = 0.f;\n        return;\n    }\n    double X0[3]", "tests/test_oracle_interp.py"),
    ("y1 from cx", INTERP, "y1 = P->focal * X1[1] / X1[2] + P->cy;", "y1 = P->focal * X1[1] / X1[2] + P->cx;",
     "tests/test_oracle_interp.py"),
]


def _planted(tmp, k, path, text, repl):
    srcs = []
    for src in oracle.SOURCES:
        body = open(src).read()
        if src == path:
            assert body.count(text) == 1, f"mutation {k}: the text must occur exactly once in {src}"
            body = body.replace(text, repl)
        dst = os.path.join(tmp, f"m{k}_" + os.path.basename(src))
        with open(dst, "w") as f:
            f.write(body)
        srcs.append(dst)
    return oracle.compile_library(srcs, os.path.join(tmp, f"m{k}_liboracle.so"))


def _run(tmp, k, mutation):
    name, path, text, repl, module = mutation
    lib = _planted(tmp, k, path, text, repl)
    env = dict(os.environ, SFF_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", module, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return name, module, r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if os.environ.get("SFF_ORACLE_LIB"):
        pytest.skip("running against a planted copy already")
    oracle.build()
    workers = max(1, min(4, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as pool:
        results = list(pool.map(lambda km: _run(str(tmp_path), *km), enumerate(MUTATIONS)))
    # exit status 1: tests ran and some failed; anything else (0 = all passed,
    # 2+ = errors) means the pin did not catch the mistake as a test failure
    missed = [(name, module, rc) for name, module, rc in results if rc != 1]
    assert not missed, missed
