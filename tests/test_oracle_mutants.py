"""The oracle's pins catch plausible mistakes.

Each mutant below is the oracle's C source with one deliberate mistake of the
kind a restatement of the paper can make (a dropped term, a wrong sign,
index or operand order, an off-by-one).  It is built into a temporary library
and the pin tests run against it in a subprocess (CPT_ORACLE_LIB); some pin
must fail.  The committed oracle is never modified."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cpt_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_rates.py", "tests/test_oracle_learned.py",
        "tests/test_stream_layout.py"]

# (name, the passage it breaks, original text, mutated text)
MUTANTS = [
    ("alg2-dropped-M0", "Alg. 2",
     "i64 M = M0 + M1 + M2;", "i64 M = M1 + M2;"),
    ("alg2-same-sign-wrong-vertex", "Alg. 2",
     "if (same_sign(u0, u1, u2) && iabs64(u2) - 1 > eb) eb = iabs64(u2) - 1;",
     "if (same_sign(u0, u1, u2) && iabs64(u1) - 1 > eb) eb = iabs64(u1) - 1;"),
    ("alg2-non-strict-ratio", "Alg. 2 (strict bound)",
     "return num > 0 ? (num - 1) / den : 0;", "return num > 0 ? num / den : 0;"),
    ("sos-first-perturbation-sign", "Alg. 1 (SoS)",
     "if (bu != 0) return bu > 0 ? -1 : 1;", "if (bu != 0) return bu > 0 ? 1 : -1;"),
    ("face-test-orientation", "Eq. 2",
     "int s20 = -o_sos_det2(p[0], p[1], p[4], p[5]);", "int s20 = o_sos_det2(p[0], p[1], p[4], p[5]);"),
    ("mesh-face-3-corner", "Sec. III-C (prism split)",
     "/* 3: (A_t, R_t+1, G_t+1)        */ {{0, 0, 0}, {1, 0, 1}, {1, 1, 1}},",
     "/* 3: (A_t, R_t+1, G_t+1)        */ {{0, 0, 0}, {1, 1, 0}, {1, 1, 1}},"),
    ("mesh-tet-face-owner", "Sec. III-C (prism split)",
     "{{0, 0, 0, 0}, {0, 0, 0, 2}, {0, 0, 0, 10}, {0, 0, 1, 8}},",
     "{{0, 0, 0, 0}, {0, 0, 0, 2}, {0, 0, 0, 10}, {0, 1, 0, 8}},"),
    ("alg4-crossed-face-ignored", "Alg. 4",
     "if (mask[vid(H, W, ot, oi, oj)] & (1u << type)) {",
     "if (0 && (mask[vid(H, W, ot, oi, oj)] & (1u << type))) {"),
    ("fixed-point-one-bit-short", "Alg. 3 (fixed point)",
     "return 23 - e;", "return 22 - e;"),
    ("lorenzo-corner-sign", "Sec. VI (3-D Lorenzo)",
     "qat(Q, H, W, t - 1, i, j - 1, c) + qat(Q, H, W, t - 1, i - 1, j - 1, c);",
     "qat(Q, H, W, t - 1, i, j - 1, c) - qat(Q, H, W, t - 1, i - 1, j - 1, c);"),
    ("quantiser-bin-width", "Sec. V (linear quantisation)",
     "i64 w = 2 * xiq + 1;", "i64 w = 2 * xiq;"),
    ("sl-downstream-trace", "Eqs. 7-8",
     "xs = clampf((float)j - uh * cfl_x, (float)(W - 1));",
     "xs = clampf((float)j + uh * cfl_x, (float)(W - 1));"),
    ("sl-u-v-swapped", "Eqs. 5-8",
     "float du = (float)g[0] * cfl_x;", "float du = (float)g[1] * cfl_x;"),
    ("sl-substep-count", "Eq. 9",
     "float nd = ceilf(dinf / 2.0f);", "float nd = ceilf(dinf / 4.0f);"),
    ("bilinear-weights-transposed", "Eq. 6",
     "float w00 = gx * gy, w10 = fx * gy, w01 = gx * fy, w11 = fx * fy;",
     "float w00 = gx * gy, w10 = gx * fy, w01 = fx * gy, w11 = fx * fy;"),
    ("mop-switch-reversed", "Sec. VI-B",
     "uint8_t m = (1000 * rs < 997 * r3) ? 1 : 0;", "uint8_t m = (1000 * r3 < 997 * rs) ? 1 : 0;"),
    ("mop-penalty-weight", "Eq. 10",
     "pen = (i64)(((u64)16 * n_fail << 32)", "pen = (i64)(((u64)8 * n_fail << 32)"),
    ("ilog2-mantissa", "Eq. 10 (entropy estimate)",
     "u64 y = ((u64)x << 31) >> e;", "u64 y = ((u64)x << 30) >> e;"),
    ("eps-prime-rounding", "Alg. 3 (eps' of the fixed-point field)",
     "double e = floor(ldexp(eps, k) - 0.5);", "double e = floor(ldexp(eps, k));"),
    ("to-fixed-floor", "Alg. 3 (fixed point)",
     "q[n] = (int32_t)rint(ldexp((double)uv[n], k));", "q[n] = (int32_t)floor(ldexp((double)uv[n], k));"),
    ("face-valid-boundary", "Sec. III-C (mesh boundary)",
     "if (tt >= T || ii >= H || jj >= W) return 0;", "if (tt >= T || ii >= H || jj > W) return 0;"),
    ("alg4-third-vertex-skipped", "Alg. 4 (every incident face)",
     "    i64 self = vid(H, W, t, i, j);\n    for (int type = 0; type < 12; ++type)\n        for (int k = 0; k < 3; ++k) {",
     "    i64 self = vid(H, W, t, i, j);\n    for (int type = 0; type < 12; ++type)\n        for (int k = 0; k < 2; ++k) {"),
    ("rk2-full-step-midpoint", "Eqs. 7-8 (midpoint)",
     "float xh = clampf((float)j - 0.5f * du, (float)(W - 1));",
     "float xh = clampf((float)j - 1.0f * du, (float)(W - 1));"),
    ("trajectory-reverse-link-dropped", "Thm. 2 (faces joined through tets)",
     "if (nb[2 * c] < 0) nb[2 * c] = a; else nb[2 * c + 1] = a;", "(void)0;"),
    ("trajectory-walk-start", "Thm. 2 (paths from their ends)",
     "if (pass == 0 && deg == 2) continue;", "if (pass == 0 && deg != 2) continue;"),
    ("net-relu-dropped", "learned predictor (ReLU after layers 1 and 2)",
     "out[((i64)co * H + i) * W + j] = relu ? (acc > 0.0f ? acc : 0.0f) : acc;",
     "out[((i64)co * H + i) * W + j] = acc;"),
    ("net-kernel-transposed", "learned predictor (3 x 3 kernel taps)",
     "acc = fmaf(bf16f(w[((co * cin + ci) * 3 + ky) * 3 + kx]), v, acc);",
     "acc = fmaf(bf16f(w[((co * cin + ci) * 3 + kx) * 3 + ky]), v, acc);"),
    ("net-clamp", "learned predictor (output clamp)",
     "d = d < -2.0f ? -2.0f : (d > 2.0f ? 2.0f : d);", "d = d < -1.0f ? -1.0f : (d > 1.0f ? 1.0f : d);"),
    ("net-parameter-layout", "learned predictor (parameter layout)",
     "const uint16_t* w2 = b1 + NET_C;", "const uint16_t* w2 = b1 + NET_C - 1;"),
    ("stream-bit-order", "reading R12 (codes most significant bit first)",
     "if ((c >> k) & 1u) words[pos >> 5] |= 1u << (31 - (pos & 31));",
     "if ((c >> k) & 1u) words[pos >> 5] |= 1u << (pos & 31);"),
    ("stream-canonical-order", "reading R12 (canonical codes)",
     "        if (len[s]) code[s] = next[len[s]]++;",
     "        if (len[s]) code[s] = next[len[s]]++ ^ 1u;"),
    ("stream-sync-offset", "reading R12 (sync points)",
     "if (x % HUFF_CHUNK == 0) put_u64(b, nbits);", "if (x % HUFF_CHUNK == 0) put_u64(b, nbits + (x > 0));"),
    ("huffman-lengths-to-heavy-leaves", "Sec. VII-E (Huffman stage)",
     "for (size_t x = 0; x < leaves; ++x) len[lv[x].sym]++;",
     "for (size_t x = 0; x < leaves; ++x) len[lv[n - 1 - x].sym]++;"),
]


def _build(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the original text must occur once"
    path_c = os.path.join(tmp, f"{name}.c")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    path_so = os.path.join(tmp, f"lib{name}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", path_so, path_c, "-lm"], check=True, capture_output=True)
    return path_so


def _run_pins(so):
    env = dict(os.environ, CPT_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


@pytest.mark.timeout(900)
def test_every_mutant_fails_a_pin(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    libs = {name: _build(str(tmp_path), name, old, new) for name, _, old, new in MUTANTS}
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(libs, ex.map(_run_pins, libs.values())))
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, {n: results[n][1] for n in survivors}


def test_unmutated_copy_passes(tmp_path):
    """Control: the same build route without a mutation passes every pin."""
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    so = _build(str(tmp_path), "control", "int o_xi_code(i64 xi)", "int o_xi_code(i64 xi)")
    rc, out = _run_pins(so)
    assert rc == 0, out
