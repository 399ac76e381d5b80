"""Planted mistakes in the oracle must each make a pin fail.

Each case replaces one fragment of `oracle/tsplat_oracle.c` (a flipped sign,
a transposed index, a dropped term, an off-by-one, a wrong constant), builds
the copy into a temporary directory with the oracle's own compiler flags,
and runs `tests/test_oracle_pins.py` against it (the oracle loads the
library that TSPLAT_ORACLE_LIB names).  A mutation that no pin notices would
mean a part of the oracle is not tied to anything outside itself.  The cases
cover the BF16 rounding, the lifting, the key-mode and FP64 projections and
their near and far planes, the tile rects, the scan, the emission, the sort
and the ranges, the compositing, the adjoints of the compositing, the
projection and the lifting, the ambiguity flags and the alternative outputs
at threshold decisions, the point z-buffer, the tight binning and its
key-mode logarithm.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tsplat_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the mistake is, fragment of the oracle source, its mutated form)
MUTATIONS = [
    ('lift f32 t sign',
     'float d1 = ry * z - t[1];',
     'float d1 = ry * z + t[1];'),
    ('lift f64 transpose',
     'mean[3 * n + i] = R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1] + R[2 * 3 + i] * d[2];',
     'mean[3 * n + i] = R[i * 3 + 0] * d[0] + R[i * 3 + 1] * d[1] + R[i * 3 + 2] * d[2];'),
    ('lift f32 quat idx',
     'Rq[1][2] = 2.0f * (y * zq - w * x);',
     'Rq[1][2] = 2.0f * (y * zq - w * y);'),
    ('lift f32 scale idx',
     'M[i][j] = rg * scale[3 * p + j];',
     'M[i][j] = rg * scale[3 * p + i];'),
    ('proj j02 sign',
     'float j00 = fx / pz, j02 = -((fx * tx) / pz2);',
     'float j00 = fx / pz, j02 = ((fx * tx) / pz2);'),
    ('proj f64 J sign',
     'double J[2][3] = {{fx / p[2], 0, -fx * tx / (p[2] * p[2])},',
     'double J[2][3] = {{fx / p[2], 0, fx * tx / (p[2] * p[2])},'),
    ('proj f64 transpose',
     'T[r][j] = J[r][0] * R[0 * 3 + j] + J[r][1] * R[1 * 3 + j] + J[r][2] * R[2 * 3 + j];',
     'T[r][j] = J[r][0] * R[j * 3 + 0] + J[r][1] * R[j * 3 + 1] + J[r][2] * R[j * 3 + 2];'),
    ('proj conic b sign',
     'conic[3 * i] = c / det; conic[3 * i + 1] = -(b / det);',
     'conic[3 * i] = c / det; conic[3 * i + 1] = (b / det);'),
    ('proj f64 conic swap',
     'conic[3 * i] = c / det; conic[3 * i + 1] = -b / det; conic[3 * i + 2] = a / det;',
     'conic[3 * i] = a / det; conic[3 * i + 1] = -b / det; conic[3 * i + 2] = c / det;'),
    ('proj disc sign',
     'float disc = fmaxf(0.1f, mid * mid - det);',
     'float disc = fmaxf(0.1f, mid * mid + det);'),
    ('proj radius 2 sigma',
     'float r = ceilf(3.0f * sqrtf(lam));',
     'float r = ceilf(2.0f * sqrtf(lam));'),
    ('proj rect +16',
     'fx1 = floorf(((mx + r) + 15.0f) / 16.0f);',
     'fx1 = floorf(((mx + r) + 16.0f) / 16.0f);'),
    ('proj lowpass dropped',
     'float a = s00 + lp, b = s01, c = s11 + lp;',
     'float a = s00, b = s01, c = s11 + lp;'),
    ('sort unstable',
     'if (ka[j] < ka[i]) { kb[o] = ka[j]; vb[o++] = va[j++]; }',
     'if (ka[j] <= ka[i]) { kb[o] = ka[j]; vb[o++] = va[j++]; }'),
    ('comp no T in weight',
     'const double w = alpha * T;',
     'const double w = alpha;'),
    ('comp stop on T',
     'int stop = Tn < in->t_min;',
     'int stop = T < in->t_min;'),
    ('comp q b sign',
     'const double q = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;',
     'const double q = -0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy;'),
    ('comp alpha clamp',
     'double alpha = e < in->alpha_max ? e : in->alpha_max;',
     'double alpha = e;'),
    ('comp last index',
     'last = (int32_t)(k - start + 1);',
     'last = (int32_t)(k - start);'),
    ('bwd S term',
     'const double dalpha = Tj * fg - S / (1.0 - alpha) + gA * Tfinal / (1.0 - alpha);',
     'const double dalpha = Tj * fg + gA * Tfinal / (1.0 - alpha);'),
    ('bwd gA sign',
     'const double dalpha = Tj * fg - S / (1.0 - alpha) + gA * Tfinal / (1.0 - alpha);',
     'const double dalpha = Tj * fg - S / (1.0 - alpha) - gA * Tfinal / (1.0 - alpha);'),
    ('bwd dmu sign',
     'd_mu[2 * j] += dq * (a * dx + b * dy);',
     'd_mu[2 * j] -= dq * (a * dx + b * dy);'),
    ('bwd dconic b',
     'd_conic[3 * j + 1] += dq * (-dx * dy);',
     'd_conic[3 * j + 1] += dq * (-0.5 * dx * dy);'),
    ('bwd dmu index',
     'd_mu[2 * j + 1] += dq * (b * dx + c * dy);',
     'd_mu[2 * j + 1] += dq * (b * dy + c * dx);'),
    ('pbwd gB sign',
     'const double ga = -gA * c * c / D2 + gB * b * c / D2 + gC * (1.0 / D - a * c / D2);',
     'const double ga = -gA * c * c / D2 - gB * b * c / D2 + gC * (1.0 / D - a * c / D2);'),
    ('pbwd gt1 swap',
     'gt1[k] = gb * VT0[k] + 2 * gcc * VT1[k];',
     'gt1[k] = gb * VT1[k] + 2 * gcc * VT0[k];'),
    ('pbwd clamp ignored',
     'gp[2] += fx * txz / (z * z) * gJ02;',
     'gp[2] += 2 * fx * p[0] / (z * z * z) * gJ02;'),
    ('pbwd offdiag double',
     'd00 += T[0][v] * T[0][u];',
     'd00 += 0;'),
    ('pbwd mean transpose',
     'gm[k] = R[0 * 3 + k] * gp[0] + R[1 * 3 + k] * gp[1] + R[2 * 3 + k] * gp[2];',
     'gm[k] = R[k * 3 + 0] * gp[0] + R[k * 3 + 1] * gp[1] + R[k * 3 + 2] * gp[2];'),
    ('pbwd mu z term',
     '-fx * p[0] / (z * z) * g_mu[2 * i] - fy * p[1] / (z * z) * g_mu[2 * i + 1]};',
     '-fx * p[0] / (z * z) * g_mu[2 * i]};'),
    ('lbwd G offdiag',
     'const double G[3][3] = {{gc[0], gc[1] / 2, gc[2] / 2}, {gc[1] / 2, gc[3], gc[4] / 2},',
     'const double G[3][3] = {{gc[0], gc[1], gc[2] / 2}, {gc[1], gc[3], gc[4] / 2},'),
    ('lbwd ray transpose',
     'gz += (Rs[0 * 3 + i] * ray[0] + Rs[1 * 3 + i] * ray[1] + Rs[2 * 3 + i] * ray[2]) * gm[i];',
     'gz += (Rs[i * 3 + 0] * ray[0] + Rs[i * 3 + 1] * ray[1] + Rs[i * 3 + 2] * ray[2]) * gm[i];'),
    ('lbwd scale factor',
     'for (int i = 0; i < 3; ++i)\n                for (int j = 0; j < 3; ++j) gM[i][j] = 2 * (G[i][0]',
     'for (int i = 0; i < 3; ++i)\n                for (int j = 0; j < 3; ++j) gM[i][j] = 1 * (G[i][0]'),
    ('lbwd quat gw sign',
     'const double gw = 2 * (-zq * gRq[0][1] + y * gRq[0][2]',
     'const double gw = 2 * (zq * gRq[0][1] + y * gRq[0][2]'),
    ('lbwd quat norm',
     'g_quat[4 * p] = (gw - w * dot) / nq;',
     'g_quat[4 * p] = gw / nq;'),
    ('lbwd gRq s',
     'gRq[k][j] = (Rs[k * 3 + 0] * gM[0][j] + Rs[k * 3 + 1] * gM[1][j] + Rs[k * 3 + 2] * gM[2][j]) * s3[j];',
     'gRq[k][j] = (Rs[0 * 3 + k] * gM[0][j] + Rs[1 * 3 + k] * gM[1][j] + Rs[2 * 3 + k] * gM[2][j]) * s3[j];'),
    ('b sign in q',
     'return dx * (a * dx + b2 * dy) + (c * dy) * dy;',
     'return dx * (a * dx - b2 * dy) + (c * dy) * dy;'),
    ('b not doubled',
     'const float b2 = 2.0f * b, ra = b / a, rc = b / c;',
     'const float b2 = b, ra = b / a, rc = b / c;'),
    ('vertex sign',
     'd = clampf_(-(ra * dy0), dx0, dx1);',
     'd = clampf_((ra * dy0), dx0, dx1);'),
    ('swap ra rc',
     'd = clampf_(-(rc * dx0), dy0, dy1);',
     'd = clampf_(-(ra * dx0), dy0, dy1);'),
    ('a c swap',
     'const float b2 = 2.0f * b, ra = b / a, rc = b / c;\n    float q',
     'const float b2 = 2.0f * b, ra = b / c, rc = b / a;\n    float q'),
    ('drop edge',
     'd = clampf_(-(rc * dx1), dy0, dy1); q = fminf(q, tight_q(a, b2, c, dx1, d));',
     ';'),
    ('inside test',
     'if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 0.0f;',
     'if (dx0 <= 0.0f && dx1 >= 0.0f) return 0.0f;'),
    ('kappa no 2',
     'const float kappa = 2.0f * orc_key_ln_f32(ratio);',
     'const float kappa = orc_key_ln_f32(ratio);'),
    ('kappa x4',
     'const float kappa = 2.0f * orc_key_ln_f32(ratio);',
     'const float kappa = 4.0f * orc_key_ln_f32(ratio);'),
    ('ln e off',
     'return (float)e * 0.693147182f + 2.0f * (t * s);',
     'return (float)(e + 1) * 0.693147182f + 2.0f * (t * s);'),
    ('ln series',
     's = s * t2 + 0.333333333f;',
     's = s * t2 + 0.5f;'),
    ('px1 no clip',
     'const float px1 = (float)(TILE * tx + TILE - 1 < W - 1 ? TILE * tx + TILE - 1 : W - 1);',
     'const float px1 = (float)(TILE * tx + TILE);'),
    ('tile origin',
     'const float px0 = (float)(TILE * tx), py0 = (float)(TILE * ty);',
     'const float px0 = (float)(TILE * tx + 1), py0 = (float)(TILE * ty);'),
    ('bit index',
     'if (qm <= thr) m |= 1u << ((ty - y0) * w + (tx - x0));',
     'if (qm <= thr) m |= 1u << ((tx - x0) * w + (ty - y0));'),
    ('emit bit',
     'const int bit = (ty - y0) * w + (tx - x0);',
     'const int bit = (tx - x0) * (y1 - y0) + (ty - y0);'),
    ('low opacity kept',
     'if (ratio >= 1.0f) {',
     'if (ratio >= 0.0f) {'),
    ('bf16 round half up',
     'u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;',
     'u = (u + 0x8000u) & 0xFFFF0000u;'),
    ('bf16 truncation',
     'u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;',
     'u = u & 0xFFFF0000u;'),
    ('zbuffer ties keep last',
     'if (bits < best[p]) {',
     'if (bits <= best[p]) {'),
    ('zbuffer pixel floor',
     'const float fu = floorf(mx + 0.5f), fv = floorf(my + 0.5f);',
     'const float fu = floorf(mx), fv = floorf(my + 0.5f);'),
    ('zbuffer far plane',
     '        if (!(pz > znear && pz < zfar)) continue;\n        const float mx = (fx * px) / pz + cx;',
     '        if (!(pz > znear)) continue;\n        const float mx = (fx * px) / pz + cx;'),
    ('scan inclusive',
     'for (int64_t i = 0; i < n; ++i) { offsets[i] = acc; acc += ntiles[i]; }',
     'for (int64_t i = 0; i < n; ++i) { acc += ntiles[i]; offsets[i] = acc - (i == 0 ? ntiles[0] : 0); }'),
    ('emit column-major tile id',
     '            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {\n                keys[k] = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | dkey[i];\n                vals[k] = (uint32_t)i;\n                ++k;\n            }\n    }\n}',
     '            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {\n                keys[k] = ((uint64_t)(uint32_t)(tx * tiles_x + ty) << 32) | dkey[i];\n                vals[k] = (uint32_t)i;\n                ++k;\n            }\n    }\n}'),
    ('ranges end off by one',
     'ranges[2 * tile + 1] = (uint32_t)(k + 1);',
     'ranges[2 * tile + 1] = (uint32_t)k;'),
    ('project far plane dropped',
     '        if (!(pz > znear && pz < zfar)) continue;\n\n        float txz',
     '        if (!(pz > znear)) continue;\n\n        float txz'),
    ('project near plane inclusive',
     '        if (!(pz > znear && pz < zfar)) continue;\n\n        float txz',
     '        if (!(pz >= znear && pz < zfar)) continue;\n\n        float txz'),
    ('alternatives skip the last subset',
     'for (int mask = 1; mask < (1 << na); ++mask) {',
     'for (int mask = 1; mask < (1 << na) - 1; ++mask) {'),
    ('alternatives alpha output',
     'out[n_alt * (C + 1) + C] = 1.0 - T;',
     'out[n_alt * (C + 1) + C] = T;'),
    ('alpha margin not flagged',
     'if (fabs(alpha - in->alpha_min) <= in->margin_alpha * in->alpha_min) {',
     'if (0 && fabs(alpha - in->alpha_min) <= in->margin_alpha * in->alpha_min) {'),
    ('T margin not flagged',
     'if (fabs(Tn - in->t_min) <= in->margin_t * in->t_min) {',
     'if (0 && fabs(Tn - in->t_min) <= in->margin_t * in->t_min) {'),
    ('flip of T ignored',
     'if (is_flipped(flips, nflips, k, DEC_T)) stop = !stop;',
     ';'),
    ('alpha skip inclusive',
     'int skip_a = alpha < in->alpha_min;',
     'int skip_a = alpha <= in->alpha_min;'),
    ('stop inclusive',
     'int stop = Tn < in->t_min;',
     'int stop = Tn <= in->t_min;'),
    ('T update before weight',
     'const double w = alpha * T;',
     'const double w = alpha * T * (1.0 - alpha);'),
]


def _caught(args):
    i, (name, old, new), tmp = args
    src = open(SRC).read()
    if src.count(old) != 1:
        return name, "fragment not found exactly once"
    c = os.path.join(tmp, f"m{i}.c")
    so = os.path.join(tmp, f"m{i}.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new))
    r = subprocess.run(["gcc", *O.CFLAGS, "-o", so, c, "-lm"], capture_output=True, text=True)
    if r.returncode:
        return name, "does not compile: " + r.stderr[-300:]
    env = dict(os.environ, TSPLAT_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    # caught: the pins ran and one failed (exit 1), or the mutated oracle
    # crashed the run (killed by a signal)
    caught = r.returncode == 1 or r.returncode < 0
    return name, None if caught else f"pins exit {r.returncode}: " + r.stdout[-300:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    jobs = [(i, m, str(tmp_path)) for i, m in enumerate(MUTATIONS)]
    with ThreadPoolExecutor(max(1, min(4, (os.cpu_count() or 2) // 2))) as ex:
        results = list(ex.map(_caught, jobs))
    missed = [(name, why) for name, why in results if why]
    assert not missed, missed
    assert len(results) >= 70
