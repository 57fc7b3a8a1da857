"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (the
host-side sanitiser run): a separate build of sj_oracle.c with both
sanitizers, loaded in a child process with the ASan runtime preloaded, runs
the filter, brute-force and grid-filtered PIP and P2P on small workloads and
the exact-predicate mode; any report fails the test."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
from oracle import oracle as O
O.use(O.build(sanitize=True))
from paper_1403_0802_gb300 import synth
w = synth.pip_tiles(n_points=3000, layer=3, grid_n=64)
P = w.polygons
mbb = O.pip_mbb(w.grid, P.verts, P.ring_off, P.poly_ring_off)
cs, ci = O.cand_csr(w.grid, mbb)
a = O.pip_grid(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off, cs, ci)
b = O.pip_brute(w.grid, w.points[:500], P.verts, P.ring_off, P.poly_ring_off)
assert (a[:500] == b).all() and (a >= 0).all()
with O.exact_predicates():
    assert (O.pip_grid(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off, cs, ci) == a).all()
w = synth.p2p_walks(n_points=3000, n_lines=2000, grid_n=64)
L = w.polylines
r = O.p2p_join(w.grid, w.points, L.verts, L.line_off, w.D)
s = O.p2p_brute(w.grid, w.points[:300], L.verts, L.line_off, w.D)
assert (r[0][:300] == s[0]).all()
pts = np.concatenate([w.points[:10], [[np.nan, 1.0], [-5.0, 3.0], [1e5, 1e5]]])
O.point_cells(w.grid, pts)
O.cell_counts(w.grid, pts)
print("sanitized ok")
""".replace("ROOT", repr(ROOT))


def test_oracle_under_asan_and_ubsan():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    libasan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not libasan or not os.path.exists(libasan):
        pytest.skip("no ASan runtime")
    env = dict(os.environ, LD_PRELOAD=libasan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", CODE], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "sanitized ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
