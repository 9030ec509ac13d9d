"""The oracle's pins catch plausible mistakes in the oracle.

Each mutant below is a copy of oracle/simplex_oracle.c with one planted
mistake of the kind a restatement of the paper could make -- a dropped term,
a wrong bound, a swapped operand or index, a wrong constant.  The copy is
compiled on the CPU and swapped in for the real oracle while the pins of
test_oracle_pins run; at least one pin must fail for every mutant.  (Mutants
that compute the same function -- e.g. swapping x1 and x2 where the domain is
symmetric in them -- are not listed: no test can tell them apart.)  Every
mutant keeps its memory accesses inside the arrays the tests pass.
"""
import ctypes

import pytest

import oracle
import test_oracle_pins as pins

# (name, text in simplex_oracle.c, replacement, which occurrence of the text)
MUTANTS = [
    ("hash: golden-ratio step off by one", "z += 0x9E3779B9u;", "z += 0x9E3779B8u;", 0),
    ("hash: second xorshift 12 instead of 13", "(z ^ (z >> 13))", "(z ^ (z >> 12))", 0),
    ("hash: second multiplier", "0xC2B2AE35u", "0xC2B2AE37u", 0),
    ("count: m = 3 strict bound", "x1 + x2 + x3 <= n; x3++) c++;", "x1 + x2 + x3 < n; x3++) c++;", 0),
    ("count: m = 4 strict bound", "x1 + x2 + x3 + x4 <= n; x4++) c++;", "x1 + x2 + x3 + x4 < n; x4++) c++;", 0),
    ("accum: assigns instead of adding", "data[x1 * D + x2] += add;", "data[x1 * D + x2] = add;", 0),
    ("accum: m = 4 drops the face x1 + ... + x4 = n",
     "x1 + x2 + x3 + x4 <= n; x4++) {\n                        data[",
     "x1 + x2 + x3 + x4 < n; x4++) {\n                        data[", 0),
    ("write: m = 2 hash of the transposed index",
     "out[lin] = oracle_splitmix32(seed ^ (uint32_t)lin);", "out[lin] = oracle_splitmix32(seed ^ (uint32_t)(x2 * D + x1));",
     0),
    ("write: m = 3 seed added instead of xor-ed",
     "out[lin] = oracle_splitmix32(seed ^ (uint32_t)lin);", "out[lin] = oracle_splitmix32(seed + (uint32_t)lin);", 1),
    ("init: threshold test not strict", "(uint32_t)lin) < threshold ? 1 : 0;", "(uint32_t)lin) <= threshold ? 1 : 0;", 0),
    ("init: row stride D + 1",
     "int64_t lin = x1 * D + x2;\n                uint8_t a", "int64_t lin = x1 * (D + 1) + x2;\n                uint8_t a", 0),
    ("step: the cell counts itself",
     "if (d1 == 0 && d2 == 0) continue;\n                        int64_t y1 = x1 + d1",
     "int64_t y1 = x1 + d1", 0),
    ("step: birth and survive swapped",
     "uint8_t next = alive ? (uint8_t)((survive >> k) & 1u) : (uint8_t)((birth >> k) & 1u);",
     "uint8_t next = alive ? (uint8_t)((birth >> k) & 1u) : (uint8_t)((survive >> k) & 1u);", 0),
    ("step: m = 3 neighbours on the face y1 + y2 + y3 = n dropped",
     "y1 + y2 + y3 <= n;", "y1 + y2 + y3 < n;", 0),
    ("step: m = 2 neighbours in column 0 dropped",
     "return y1 >= 0 && y2 >= 0 && y1 + y2 <= n;", "return y1 >= 0 && y2 >= 1 && y1 + y2 <= n;", 0),
    ("step: m = 3 neighbour offsets -1, 0 only", "for (int d3 = -1; d3 <= 1; d3++)", "for (int d3 = -1; d3 < 1; d3++)", 0),
    ("run: initial live count dropped", "live[0] = c;", "live[0] = 0;", 0),
    ("run: first step reads the wrong buffer",
     "const uint8_t *src = (s % 2 == 1) ? a : b;", "const uint8_t *src = (s % 2 == 0) ? a : b;", 0),
    ("cells: alive read from the transposed cell",
     "alive = in[x[0] * D + x[1]];", "alive = in[x[1] * D + x[0]];", 0),
    ("block indicator: m = 2 cells on the face x1 + x2 = n dropped",
     "x1 + x2 <= n; x2++)\n                ind[", "x1 + x2 < n; x2++)\n                ind[", 0),
    ("edm: point j = x2 instead of n - x2", "*b = points + (n - x2) * dim;", "*b = points + x2 * dim;", 0),
    ("edm: last coordinate dropped", "for (int k = 0; k < dim; k++) {", "for (int k = 0; k < dim - 1; k++) {", 0),
    ("edm: square root missing", "out[x1 * D + x2] = sqrt(s);", "out[x1 * D + x2] = s;", 0),
    ("edm cells: coordinates swapped",
     "const int64_t x1 = coords[2 * i], x2 = coords[2 * i + 1];",
     "const int64_t x2 = coords[2 * i], x1 = coords[2 * i + 1];", 0),
]


def _pin_calls():
    """The pins, each with fixed arguments (the parametrized ones at a few cases)."""
    calls = [(f"splitmix32_inverts({x})", pins.test_splitmix32_inverts_to_counter, (x,))
             for x in (0, 1, 0x12345678, 0xFFFFFFFF)]
    calls += [(f"cell_count_closed_form(m={m})", pins.test_cell_count_closed_form, (m,)) for m in (1, 2, 3, 4)]
    calls += [("cell_count_degenerate", pins.test_cell_count_degenerate, ())]
    calls += [(f"accum{c}", pins.test_accum_adds_once_to_every_domain_cell, c) for c in ((2, 9), (3, 6), (4, 4))]
    calls += [(f"write{c}", pins.test_write_support_and_values, c) for c in ((2, 7), (3, 5), (4, 4))]
    calls += [("init_rule_and_rate", pins.test_init_matches_threshold_rule_and_rate, ()),
              ("init_threshold_strict", pins.test_init_threshold_is_strict, ()),
              ("life_hand_worked", pins.test_life_hand_worked_delta2, ()),
              ("life_still", pins.test_life_block_and_beehive_are_still, ()),
              ("life_blinker", pins.test_life_blinker_period_two, ()),
              ("life_glider", pins.test_life_glider_moves_one_diagonal_per_four_steps, ()),
              ("all_dead", pins.test_all_dead_stays_dead_and_outside_never_lives, ()),
              ("outside_content", pins.test_ca_step_ignores_outside_content, ()),
              ("run_live", pins.test_ca_run_live_counts_are_popcounts, ()),
              ("cells_vs_step", pins.test_ca_cells_agrees_with_whole_step, ())]
    calls += [(f"shift_sum_2d{r}{n}", pins.test_ca_step_2d_matches_shift_sum, (r, n))
              for r in pins.RULES_2D for n in (5, 17)]
    calls += [(f"shift_sum_3d{r}{n}", pins.test_ca_step_3d_matches_shift_sum, (r, n))
              for r in pins.RULES_3D for n in (3, 8)]
    calls += [(f"block_indicator{c}", pins.test_block_indicator_closed_form, c)
              for c in ((2, 100, 16), (2, 64, 16), (3, 40, 8), (3, 48, 8), (4, 30, 8), (4, 32, 8))]
    calls += [("edm_pythagorean", pins.test_edm_pythagorean_points, ()),
              ("edm_cells", pins.test_edm_cells_agree_with_whole_matrix, ())]
    calls += [(f"edm_cdist{c}", pins.test_edm_matches_scipy_cdist, c) for c in ((30, 3), (57, 16))]
    return calls


def _failing_pins(monkeypatch, lib):
    failed = []
    with monkeypatch.context() as mp:
        mp.setattr(oracle, "_lib", lib)
        for name, fn, args in _pin_calls():
            try:
                fn(*args)
            except pytest.skip.Exception:
                pass
            except Exception:  # an assertion, or an error the mistake causes
                failed.append(name)
    return failed


@pytest.fixture(scope="module")
def source():
    with open(oracle._SRC) as f:
        return f.read()


def _mutate(src, old, new, k):
    at = -1
    for _ in range(k + 1):
        at = src.find(old, at + 1)
        assert at >= 0, f"mutation site not found: {old!r} (occurrence {k})"
    return src[:at] + new + src[at + len(old):]


def test_unmutated_oracle_passes_every_pin(monkeypatch, source, tmp_path):
    """The harness itself: the real source, compiled the same way, fails no pin."""
    src = tmp_path / "same.c"
    src.write_text(source)
    lib = oracle.configure(ctypes.CDLL(oracle.compile_source(str(src), str(tmp_path / "libsame.so"))))
    assert _failing_pins(monkeypatch, lib) == []


@pytest.mark.parametrize("name,old,new,k", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(monkeypatch, source, tmp_path, name, old, new, k):
    src = tmp_path / "mutant.c"
    src.write_text(_mutate(source, old, new, k))
    lib = oracle.configure(ctypes.CDLL(oracle.compile_source(str(src), str(tmp_path / "libmutant.so"))))
    assert _failing_pins(monkeypatch, lib), f"no pin fails for the mutant: {name}"
