"""The oracle's pins have teeth: each plausible slip, planted in a copy of the
oracle (on the CPU, never in the product), makes `test_oracle_pins.py` fail.

Every case copies `oracle/` to a temporary directory, applies one textual
change to `oracle.c` or to the Python wrapper, and runs the pin suite in a
subprocess whose import path puts the copy first (the copy builds its own
liboracle.so).  A mutation the pins let through fails this test.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file in oracle/, text, replacement)
MUTATIONS = [
    ("SDDMM gathers B by the row index", "oracle.c",
     "elem(dtb, B, j * ldb + k, b_scale, j);\n                acc", "elem(dtb, B, i * ldb + k, b_scale, j);\n                acc"),
    ("second value factor dropped", "oracle.c", "    if (vals2) s *= vals2[e];", ""),
    ("round-half-even tie goes to odd", "oracle.c",
     "pick = (lo & 1) ? lo + 1 : lo;", "pick = (lo & 1) ? lo : lo + 1;"),
    ("SpMM^T reads Y by the column", "oracle.c",
     "elem(dty, Y, i * ldy + k, y_scale, i)", "elem(dty, Y, j * ldy + k, y_scale, i)"),
    ("merge path takes the nonzero first on a tie", "oracle.c",
     "if (r < M && rowptr[r + 1] <= e) r++;", "if (r < M && rowptr[r + 1] < e) r++;"),
    ("transpose not stable", "oracle.c",
     "int64_t p = cursor[colidx[e]]++;", "int64_t p = --cursor[colidx[e] + 1];"),
    ("E4M3 row scale ignored", "oracle.c", "    if (scale) v *= (double)scale[row];", ""),
    ("SpMM overwrites instead of accumulating", "oracle.c",
     "c[k] += abs_mode ? fabs(t) : t;", "c[k] = abs_mode ? fabs(t) : t;"),
    ("E4M3 subnormal exponent off by one", "oracle.c",
     "v = ldexp((double)m / 8.0, -6);", "v = ldexp((double)m / 8.0, -7);"),
    ("E4M3 scale uses 240", "oracle.c", "amax / 448.0f", "amax / 240.0f"),
    ("FusedMM lse without the log", "oracle.c", "m + log(l) : -INFINITY", "m + l : -INFINITY"),
    ("FusedMM softmax not normalised", "oracle.c", "exp(sc - m) / l : sc", "exp(sc - m) : sc"),
    ("FusedMM score drops the scale", "oracle.c", "*score = scale * sv * dot;", "*score = sv * dot;"),
    ("FusedMM head slices overlap", "oracle.c", "int64_t k0 = h * D;", "int64_t k0 = h;"),
    ("FusedMM gradient drops the softmax row term", "__init__.py",
     "g = w * (dw - rowsum[rows])", "g = w * dw"),
    ("FusedMM gradient drops W^T dY", "__init__.py", "+ spmm_t(rowptr, colidx, N, dY[:, sl], w)", ""),
    ("FusedMM gradient drops the scale", "__init__.py", "c = scale * g", "c = g"),
]

_RUNNER = (
    "import sys; sys.path[:0] = [{copy!r}, {root!r}]\n"
    "import pytest\n"
    "sys.exit(pytest.main([{pins!r}, '-q', '-x', '-p', 'no:cacheprovider']))\n"
)


def _run_mutant(tmp, idx, name, fname, old, new):
    base = os.path.join(tmp, f"m{idx}")
    dst = os.path.join(base, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    path = os.path.join(dst, fname)
    src = open(path).read()
    assert src.count(old) >= 1, f"{name}: anchor text not found in {fname}"
    open(path, "w").write(src.replace(old, new, 1))
    runner = _RUNNER.format(copy=base, root=ROOT, pins=os.path.join(ROOT, "tests", "test_oracle_pins.py"))
    r = subprocess.run([sys.executable, "-c", runner], capture_output=True, text=True, timeout=600, cwd=base)
    return name, r.returncode, r.stdout[-400:]


def test_every_planted_slip_is_caught(tmp_path):
    # control: an unchanged copy passes, so the harness runs the copy's pins
    name, rc, out = _run_mutant(str(tmp_path), "control", "unchanged copy", "oracle.c", "int oracle_", "int oracle_")
    assert rc == 0, out
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda a: _run_mutant(str(tmp_path), *a),
                              [(i, *m) for i, m in enumerate(MUTATIONS)]))
    missed = [name for name, rc, _ in results if rc == 0]
    assert not missed, f"pins let these through: {missed}"
    # a run that failed for another reason (the copy did not build or import)
    # would also give a non-zero code: every run must have reached the pins
    for name, rc, out in results:
        assert "failed" in out or "error" in out.lower(), (name, out)
