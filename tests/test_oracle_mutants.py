"""The pins must reject an oracle with a plausible mistake planted in it.

Each mutant is a copy of oracle/sfe_oracle.c with one textual change (a
dropped term, a flipped comparison, a transposed operand, a wrong index or
sign), compiled on the CPU into a temporary library. The quick battery below
(the same checks as test_oracle_pins, at smaller sizes) must fail on every
mutant and pass on the real oracle. No mutant reads outside its buffers.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "sfe_oracle.c")

# (name, old text, new text, occurrences to replace: 0 = all)
MUTANTS = [
    # range edges: the last target or query position, the last base of a side
    ("last_target_position_dropped", "int64_t nt = tlen - p->span + 1;",
     "int64_t nt = tlen - p->span;", 1),
    ("last_query_position_dropped", "for (int64_t q = 0; q + p->span <= qlen; q++) {",
     "for (int64_t q = 0; q + p->span < qlen; q++) {", 1),
    ("right_side_stops_one_short", "while (t + span + n < tlen && q + span + n < qlen) {",
     "while (t + span + n + 1 < tlen && q + span + n < qlen) {", 1),
    ("left_side_stops_one_short", "while (t - 1 - n >= 0 && q - 1 - n >= 0) {",
     "while (t - 1 - n >= 1 && q - 1 - n >= 0) {", 1),
    # seed pattern parsing: the first care position lost
    ("first_care_position_dropped", "            p->care[p->weight++] = i;",
     "            if (i > 0) p->care[p->weight++] = i;", 1),
    ("xdrop_ge", "if (best - sum > X)", "if (best - sum >= X)", 0),
    ("latest_argmax", "if (sum > best) {", "if (sum >= best) {", 0),
    ("transversion_tolerated", "k ^ (2u << (2 * (p->weight - j)))",
     "k ^ (1u << (2 * (p->weight - j)))", 0),
    ("probe_dropped", "int nprobe = transition ? 1 + p->weight : 1;",
     "int nprobe = transition ? p->weight : 1;", 0),
    ("complement_dropped", "out[i] = (uint8_t)(q[n - 1 - i] ^ 3);",
     "out[i] = (uint8_t)(q[n - 1 - i]);", 0),
    ("transposed_operand", "sum += M[T[t + span + n] * 4 + Qs[q + span + n]];",
     "sum += M[Qs[q + span + n] * 4 + T[t + span + n]];", 0),
    ("skip_le", "if (t < E)\n                continue; /* inside",
     "if (t <= E)\n                continue; /* inside", 0),
    ("span_term_dropped", "for (int k = 0; k < span; k++)", "for (int k = 1; k < span; k++)", 0),
    ("left_starts_on_seed", "sum += M[T[t - 1 - n] * 4 + Qs[q - 1 - n]];",
     "sum += M[T[t - n] * 4 + Qs[q - n]];", 0),
    ("mask_end_without_span", "E = t + p->span + e.rext;", "E = t + e.rext;", 1),
    ("hsp_start_sign", "o.tpos = (int32_t)(t - e.lext);", "o.tpos = (int32_t)(t + e.lext);", 0),
    ("cells_without_span", "r->st.cells += p->span + e.lscored + e.rscored;",
     "r->st.cells += e.lscored + e.rscored;", 1),
    ("left_max_not_reset", "sum = best = bestlen = n = 0;", "sum = bestlen = n = 0;", 0),
    ("strand_label_swapped", "e = walk(T, tlen, Qs, qlen, s, &h,", "e = walk(T, tlen, Qs, qlen, 1 - s, &h,", 0),
    ("two_transitions_in_predicate", "if (transition && (a ^ b) == 2 && !used) {",
     "if (transition && (a ^ b) == 2) {", 0),
    ("skip_state_not_reset_per_diagonal", "int64_t E = INT64_MIN;\n        for (; i < h->n",
     "static int64_t E = INT64_MIN;\n        for (; i < h->n", 0),
]


def _safe(fn, *args) -> bool:
    """A check that raises on a broken oracle counts as a rejection."""
    try:
        r = fn(*args)
        return True if r is None else bool(r)
    except Exception:
        return False


def battery() -> dict:
    return {
        "hand": _safe(lambda: all(pins.check_hand_case(c) for c in pins._hand_cases())),
        "hits": _safe(pins.check_hits_bruteforce, 7, 1200, 1000),
        "hits_identical": _safe(pins.check_hits_adversarial, "identical"),
        "xdrop": _safe(pins.check_xdrop_exhaustive, 3, None, 910, 80),
        "xdrop_asym": _safe(pins.check_xdrop_exhaustive, 1, pins._rand_asym_scores(1), 300, 80),
        "serial": _safe(pins.check_serial_loop, 4, 1500, 1400),
        "strand": _safe(pins.check_strand_symmetry, 6),
        "swap": _safe(pins.check_swap_symmetry, 8, pins._rand_asym_scores(8)),
        "diagonal": _safe(pins.test_run_diagonal_agrees_with_run),
    }


def _mutant_source(old, new, count):
    src = open(SRC).read()
    n = src.count(old)
    assert n >= 1, f"mutation site not found: {old!r}"
    return src.replace(old, new) if count == 0 else src.replace(old, new, count)


def test_battery_passes_on_the_oracle():
    res = battery()
    assert all(res.values()), res


@pytest.mark.parametrize("name,old,new,count", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new, count):
    src = tmp_path / f"{name}.c"
    src.write_text(_mutant_source(old, new, count))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-w", "-o", str(lib), str(src)],
                   check=True)
    with oracle.use_library(str(lib)):
        res = battery()
    assert not all(res.values()), f"mutant {name} survived every pin: {res}"
