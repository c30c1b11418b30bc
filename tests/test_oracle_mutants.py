"""The pins must reject an oracle with a plausible mistake planted in it.

Each mutant is a copy of oracle/sfe_oracle.c with one textual change (a
dropped term, a flipped comparison, a transposed operand, a wrong index or
sign), compiled on the CPU into a temporary library. The quick battery below
(the same checks as test_oracle_pins, at smaller sizes) must fail on every
mutant and pass on the real oracle. No mutant reads outside its buffers.

The battery runs in two forms: the serial oracle, and the multi-threaded
form (or_run_par) with small query tiles, so that diagonals cross tiles and
the carried skip state matters. A mutant in code both forms share must be
rejected in both; a mutant in code only one form runs, in that form.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "sfe_oracle.c")

SERIAL, PARALLEL = "serial", "parallel"
BOTH = (SERIAL, PARALLEL)
PAR_QTILE, PAR_THREADS = 97, 3  # tiles of 97 query positions on 3 threads

# (name, old text, new text, occurrences to replace: 0 = all[, forms that must reject it])
MUTANTS = [
    # range edges: the last target or query position, the last base of a side
    ("last_target_position_dropped", "int64_t npos = tlen - p->span + 1;",
     "int64_t npos = tlen - p->span;", 1),
    ("last_query_position_dropped", "for (int64_t q = q0; q + p->span <= qlen && q < q1; q++) {",
     "for (int64_t q = q0; q + p->span < qlen && q < q1; q++) {", 1),
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
    ("strand_label_swapped", "walk(T, tlen, Qs, qlen, s, ", "walk(T, tlen, Qs, qlen, 1 - s, ", 0),
    ("two_transitions_in_predicate", "if (transition && (a ^ b) == 2 && !used) {",
     "if (transition && (a ^ b) == 2) {", 0),
    # the serial form starts every diagonal without a masking state; the
    # parallel form reads each diagonal's state from the carry array instead
    ("skip_state_not_reset_per_diagonal",
     "int64_t E = Ecarry ? Ecarry[d - dbase] : INT64_MIN;\n        for (; i < nh",
     "static int64_t E = INT64_MIN;\n        if (Ecarry) E = Ecarry[d - dbase];\n"
     "        for (; i < nh", 0, (SERIAL,)),
    # parallel form only: the masking state is not carried to the next query
    # tile, the last query position of every tile is lost, or two probe runs
    # of one tile overlap by a position
    ("carry_not_written_back", "        if (Ecarry)\n            Ecarry[d - dbase] = E;\n", "\n",
     1, (PARALLEL,)),
    ("tile_end_dropped", "const int64_t q1 = q0 + qtile < nq ? q0 + qtile : nq;",
     "const int64_t q1 = q0 + qtile < nq ? q0 + qtile - 1 : nq;", 1, (PARALLEL,)),
    ("probe_runs_overlap", "b = a + qrun < q1 ? a + qrun : q1;",
     "b = a + qrun + 1 < q1 ? a + qrun + 1 : q1;", 1, (PARALLEL,)),
    # the index stride: every position's key at a sampled slot, or no stride
    # test when a diagonal is walked position by position
    ("step_key_from_wrong_position", "tab[j].key = seed_key(T, j * p->step, p);",
     "tab[j].key = seed_key(T, j, p);", 1),
    ("step_ignored_on_one_diagonal", "if (t % step != 0 || !or_is_hit(",
     "if (!or_is_hit(", 1, (SERIAL,)),
]


def _safe(fn, *args) -> bool:
    """A check that raises on a broken oracle counts as a rejection."""
    try:
        r = fn(*args)
        return True if r is None else bool(r)
    except Exception:
        return False


def battery(form: str = SERIAL) -> dict:
    if form == PARALLEL:
        with oracle.use_parallel(PAR_QTILE, PAR_THREADS):
            return battery(SERIAL)
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
        "hits_step": _safe(pins.check_hits_bruteforce, 13, 1500, 1300, pins.P19, True, 0.5, 3),
        "diagonal_step": _safe(pins.test_run_diagonal_with_step_agrees_with_run),
    }


def _mutant_source(old, new, count):
    src = open(SRC).read()
    n = src.count(old)
    assert n >= 1, f"mutation site not found: {old!r}"
    return src.replace(old, new) if count == 0 else src.replace(old, new, count)


@pytest.mark.parametrize("form", BOTH)
def test_battery_passes_on_the_oracle(form):
    res = battery(form)
    assert all(res.values()), res


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, mutant):
    name, old, new, count = mutant[:4]
    forms = mutant[4] if len(mutant) > 4 else BOTH
    src = tmp_path / f"{name}.c"
    src.write_text(_mutant_source(old, new, count))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-w", "-o",
                    str(lib), str(src)], check=True)
    with oracle.use_library(str(lib)):
        for form in forms:
            res = battery(form)
            assert not all(res.values()), f"mutant {name} survived every pin ({form}): {res}"
