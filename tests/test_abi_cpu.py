"""The C-ABI library loads on a machine without a GPU and exports every
function include/sfe.h declares; host-only calls work; the product package
never reaches the oracle. No compute call is made here."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2606_06811_gb300 import build
    return build.build()


def declared() -> list[str]:
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sfe_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_every_exported_c_symbol_is_declared(built):
    """The reverse of the check above: the library exports no sfe_* C function
    that include/*.h does not declare (names from the symbol table)."""
    import shutil
    import subprocess
    if not shutil.which("nm"):
        pytest.skip("no nm")
    out = subprocess.check_output(["nm", "-D", "--defined-only", built]).decode().split("\n")
    exported = {f[2] for f in (l.split() for l in out) if len(f) == 3 and f[1] == "T"
                and f[2].startswith("sfe_")}
    assert exported and exported <= set(declared()), sorted(exported - set(declared()))


def test_host_only_calls(built):
    import paper_2606_06811_gb300 as P
    p = P.default_params()
    assert p.xdrop == 910 and p.hsp_thresh == 3000 and p.strands == 3
    assert p.seed_pattern == b"1110100110010101111"
    assert P.lib().sfe_strerror(-1) == b"invalid argument"


def test_product_path_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_06811_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\bimport\s+oracle|from\s+oracle|oracle/", txt), f


def test_autotune_candidates_skip_meaningless_combinations():
    from paper_2606_06811_gb300 import autotune, sfe
    cs = autotune.candidates(autotune.DEFAULT_SPACE)
    two = [c for c in cs if c["walk_mode"] == sfe.WALK_TWO_LAUNCHES]
    per = [c for c in cs if c["walk_mode"] == sfe.WALK_PERSISTENT]
    spec = [c for c in cs if c["walk_mode"] == sfe.WALK_SPECULATIVE]
    assert len(two) == 3 and all("walk_chunk" not in c for c in two)
    assert all(c["walk_schedule"] == sfe.SCHED_NATURAL for c in two + spec)
    assert len(per) == 3 * 2 * 2
    assert sorted(c["spec_window"] for c in spec) == [1, 4, 32]
    assert all("lane_cap" not in c and "walk_chunk" not in c for c in spec)
    assert all("spec_window" not in c for c in two + per)
    assert len(cs) == len(two) + len(per) + len(spec)
    assert len({tuple(sorted(c.items())) for c in cs}) == len(cs)


def _c_layout(struct: str, fields: list[str], tmp) -> dict:
    """sizeof and offsetof of a struct of include/sfe.h, from a C compiler."""
    import subprocess
    lines = [f'printf("size %zu\\n", sizeof({struct}));']
    lines += [f'printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"sfe.h\"\nint main(void){" + \
        "".join(lines) + "return 0;}\n"
    c = tmp / "layout.c"
    c.write_text(src)
    exe = tmp / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    return {k: int(v) for k, v in (l.split() for l in out if l)}


@pytest.mark.parametrize("name", ["Params", "Stats", "YdropParams", "YdropStats"])
def test_ctypes_mirrors_match_the_c_layout(name, tmp_path):
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    from paper_2606_06811_gb300 import sfe
    cls = getattr(sfe, name)
    struct = {"Params": "sfe_params", "Stats": "sfe_stats", "YdropParams": "sfe_ydrop_params",
              "YdropStats": "sfe_ydrop_stats"}[name]
    fields = [f for f, _ in cls._fields_]
    lay = _c_layout(struct, fields, tmp_path)
    assert lay["size"] == ctypes.sizeof(cls)
    for f in fields:
        assert lay[f] == getattr(cls, f).offset, f


def test_committed_box_index_answers_like_a_scan_of_every_box():
    """The gapped stage's index of committed boxes (a grid of 1024-base cells
    per strand, with a short list for boxes spanning many cells) against a
    scan of every box: small, empty, huge and edge-touching boxes on both
    strands, queries inside, outside and on every box edge."""
    import numpy as np
    from paper_2606_06811_gb300 import sfe
    rng = np.random.default_rng(7)
    rows = []
    for _ in range(400):  # small and medium boxes
        s = int(rng.integers(0, 2))
        t0, q0 = int(rng.integers(0, 200_000)), int(rng.integers(0, 200_000))
        w, h = int(rng.integers(0, 3000)), int(rng.integers(0, 3000))
        rows.append((s, t0, t0 + w, q0, q0 + h, 5000))
    rows.append((0, 10_000, 150_000, 20_000, 170_000, 9))  # spans far more than 4096 cells
    rows.append((1, 0, 120_000, 0, 90_000, 9))
    rows.append((0, 5_000, 5_000, 6_000, 9_000, 1))        # empty: contains nothing
    rows.append((1, 1023, 1025, 2047, 2049, 1))            # across cell edges
    B = np.array(rows, dtype=np.int32)
    Q = [(int(rng.integers(0, 2)), int(rng.integers(0, 210_000)), int(rng.integers(0, 210_000)))
         for _ in range(20_000)]
    for s, t0, t1, q0, q1, _ in rows[-4:] + rows[:50]:
        for t in (t0 - 1, t0, t1 - 1, t1):
            for q in (q0 - 1, q0, q1 - 1, q1):
                if t >= 0 and q >= 0:
                    Q.append((s, t, q))
    Q = np.array(Q, dtype=np.int32)
    got = sfe.test_committed_boxes(B, Q)
    want = np.zeros(len(Q), dtype=bool)
    for s, t0, t1, q0, q1, _ in rows:
        want |= (Q[:, 0] == s) & (t0 <= Q[:, 1]) & (Q[:, 1] < t1) & (q0 <= Q[:, 2]) & (Q[:, 2] < q1)
    assert np.array_equal(got, want)
    assert want.sum() > 1000 and (~want).sum() > 1000
    assert sfe.test_committed_boxes(B[:0], Q[:5]).sum() == 0
