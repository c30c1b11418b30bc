"""The gapped-stage pins must reject an oracle with a plausible mistake in its
Y-drop extension, its anchors, its order, its containment test or its
speculative commit (each mutant is a copy of oracle/sfe_oracle.c with one
textual change, compiled on the CPU). No mutant reads outside its buffers."""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
from tests import test_oracle_ydrop as yp

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "sfe_oracle.c")

MUTANTS = [
    ("stop_at_first_empty_antidiagonal", "if (L1 > R1 && L2 > R2)", "if (L1 > R1)", 1),
    ("gap_extend_dropped", "int32_t a = E1[i - lo1] - gext,", "int32_t a = E1[i - lo1],", 1),
    ("open_without_extend", "b = H1[i - lo1] - gopen - gext;", "b = H1[i - lo1] - gopen;", 1),
    ("ydrop_strict", "(int64_t)h < best - Y", "(int64_t)h <= best - Y", 1),
    ("latest_best_cell", "if (h > dbest) {", "if (h >= dbest) {", 1),
    ("transposed_substitution", "M[tbase(T, t0, dir, i) * 4 + tbase(Q, q0, dir, j)]",
     "M[tbase(Q, q0, dir, j) * 4 + tbase(T, t0, dir, i)]", 1),
    ("band_one_short", "chi = clo + band - 1;", "chi = clo + band - 2;", 1),
    ("diagonal_from_anti_diagonal_d1", "i - 1 >= lo2 && i - 1 <= hi2 && H2[i - 1 - lo2] > OR_YNEG)\n"
     "                dg = H2[i - 1 - lo2]", "i - 1 >= lo2 && i - 1 <= hi2 && H2[i - 1 - lo2] > OR_YNEG)\n"
     "                dg = H2[i - 1 - lo2] - 1", 1),
    ("anchor_at_hsp_start", "int64_t ta = h->tpos + h->len / 2, qa = h->qpos + h->len / 2;",
     "int64_t ta = h->tpos, qa = h->qpos;", 0),
    ("order_by_increasing_score", "if (a->score != b->score) return a->score > b->score ? -1 : 1;",
     "if (a->score != b->score) return a->score < b->score ? -1 : 1;", 1),
    ("containment_end_inclusive", "t < c[k].tend && c[k].qstart <= q", "t <= c[k].tend && c[k].qstart <= q", 1),
    ("commit_below_threshold", "if (ext[b].score >= thresh)", "if (ext[b].score >= thresh - 100000)", 1),
    ("no_commit_check_inside_a_batch", "if (b > 0 && contained(com, ncom, h->strand, ta, qa)) {",
     "if (0 && contained(com, ncom, h->strand, ta, qa)) {", 1),
]


def _safe(fn, *args) -> bool:
    try:
        r = fn(*args)
        return True if r is None else bool(r)
    except Exception:
        return False


def battery() -> dict:
    return {
        "bruteforce": _safe(yp.check_half_bruteforce, 1, 16),
        "ties": _safe(yp.check_ties),
        "xdrop": _safe(yp.check_gap_free_is_xdrop, 2, 20),
        "insertion": _safe(yp.check_insertion_case),
        "swap": _safe(yp.check_swap, 4),
        "setwise": _safe(yp.check_band_and_pruning_setwise, 7, 18),
        "batches": _safe(yp.check_batches_equal_serial, 5, (1, 3, 1000)),
        "planted": _safe(yp.check_planted_segments_one_alignment_each, 6),
        "stage": _safe(yp.check_stage_restated, 8, 6000),
    }


def test_battery_passes_on_the_oracle():
    res = battery()
    assert all(res.values()), res


@pytest.mark.parametrize("name,old,new,count", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new, count):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old!r}"
    src = src.replace(old, new) if count == 0 else src.replace(old, new, count)
    (tmp_path / "m.c").write_text(src)
    lib = tmp_path / "libm.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-w", "-o",
                    str(lib), str(tmp_path / "m.c")], check=True)
    with oracle.use_library(str(lib)):
        res = battery()
    assert not all(res.values()), f"mutant {name} survived every pin: {res}"
