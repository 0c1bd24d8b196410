"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (an
off-by-one bin, the other tie rule, a dropped term in the First recurrence,
a wrong index, the other bit order, ...), builds it, and runs the pins of
test_oracle_pins.py against it in a child process (a mutant may corrupt
memory).  Every mutant must fail at least one pin, and the unaltered source
must pass all of them in the same harness."""
import json
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (name, text in huff_oracle.c, mistaken replacement)
MUTANTS = [
    ("histogram_off_by_one_bin", "hist[s] += 1;", "hist[(s + 1) % nbins] += 1;"),
    ("joined_node_first_on_ties", "take_leaf = leaf[lh].w <= iw[ih];", "take_leaf = leaf[lh].w < iw[ih];"),
    ("leaves_by_descending_id", "return x->id < y->id ? -1 : (x->id > y->id);",
     "return x->id > y->id ? -1 : (x->id < y->id);"),
    ("heap_joined_before_leaf", "if (a->kind != b->kind) return a->kind < b->kind;",
     "if (a->kind != b->kind) return a->kind > b->kind;"),
    ("first_without_rounding_up", "first[l] = (first[l + 1] + count[l + 1] + 1) >> 1;",
     "first[l] = (first[l + 1] + count[l + 1]) >> 1;"),
    ("entry_wrong_index", "entry[l + 1] = entry[l] + count[l];", "entry[l + 1] = entry[l] + count[l + 1];"),
    ("codes_in_descending_id", "code[k] = first[l] + next[l];", "code[k] = first[l] + count[l] - 1 - next[l];"),
    ("codeword_lsb_first", "for (int b = (int)l - 1; b >= 0; b--) {\n            uint64_t w = p >> 5;",
     "for (int b = 0; b < (int)l; b++) {\n            uint64_t w = p >> 5;"),
    ("unit_codeword_lsb_first", "for (int b = (int)l - 1; b >= 0; b--) {\n            if (p / (uint64_t)W",
     "for (int b = 0; b < (int)l; b++) {\n            if (p / (uint64_t)W"),
    ("word_lsb_first", "out[w] |= bit << (31 - (p & 31));", "out[w] |= bit << (p & 31);"),
    ("chunk_offset_after_symbol", "if (i % chunk == 0) chunk_bit_offset[c++] = p;",
     "if (i % chunk == 0) chunk_bit_offset[c++] = p + len[load_sym(sym, i, width) % nbins];"),
    ("decode_entry_off_by_one", "uint32_t s = sorted_syms[entry[l] + (v - first[l])];",
     "uint32_t s = sorted_syms[entry[l] + (v - first[l]) + (l > 1)];"),
    ("single_symbol_length_two", "if (m == 1) { len[leaf[0].id] = 1; free(leaf); return 1; }",
     "if (m == 1) { len[leaf[0].id] = 2; free(leaf); return 2; }"),
    ("unit_lsb_first", "uint32_t k = (uint32_t)(W - 1 - (int)(p % (uint64_t)W));",
     "uint32_t k = (uint32_t)(p % (uint64_t)W);"),
    ("aligned_offsets_in_bits", "offs[c++] = aligned ? p / (uint64_t)W : p;", "offs[c++] = p;"),
    ("aligned_stream_not_padded_at_end", "    if (aligned) p = (p + (uint64_t)W - 1) / (uint64_t)W * (uint64_t)W;\n    offs[c]",
     "    offs[c]"),
    ("dense_form_padded_too", "if (aligned) p = (p + (uint64_t)W - 1) / (uint64_t)W * (uint64_t)W;   /* next unit boundary */",
     "p = (p + (uint64_t)W - 1) / (uint64_t)W * (uint64_t)W;"),
]

RUNNER = textwrap.dedent('''
    import ctypes, json, sys, traceback
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle
    oracle._lib = oracle._bind(ctypes.CDLL(sys.argv[1]))
    import test_oracle_pins as P
    checks = [
        ("golden", lambda: [P.test_golden_fixture(p) for p in P.FIXTURES]),
        ("bincount", lambda: P.test_histogram_matches_bincount(2, 1024)),
        ("brute_force", lambda: [P.test_lengths_brute_force_optimal(n) for n in (3, 5)]),
        ("formulations", lambda: [P.test_lengths_two_formulations_and_bounds(nb, k)
                                  for nb, k in ((17, "ties"), (256, "zipf"), (1024, "uniform"))]),
        ("edge_cases", lambda: P.test_lengths_edge_cases()),
        ("canonical", lambda: [P.test_canonical_properties(k) for k in ("ties", "zipf")]),
        ("canonical_incomplete", lambda: P.test_canonical_incomplete_lengths()),
        ("concatenation", lambda: [P.test_encode_matches_string_concatenation(n, c)
                                   for n, c in ((1025, 3), (5000, 10))]),
        ("round_trip", lambda: P.test_round_trip_synthetic_fields()),
        ("units", lambda: [P.test_encode_format_matches_string_definition(W, a, n, c)
                           for W in (8, 16) for a in (False, True) for n, c in ((37, 3), (1025, 6))]),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(name)
    print(json.dumps(failed))
''')


def _build(src_text, tmp_path, name):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(c)])
    return str(so)


def _run_pins(lib, tmp_path):
    runner = tmp_path / "run_pins.py"
    runner.write_text(RUNNER.format(root=ROOT, tests=HERE))
    r = subprocess.run([sys.executable, str(runner), lib], capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return None          # the mutant crashed the pins' process: caught too
    return json.loads(r.stdout.strip().splitlines()[-1])


def _source():
    with open(os.path.join(ROOT, "oracle", "huff_oracle.c")) as f:
        return f.read()


def test_unaltered_oracle_passes_every_pin(tmp_path):
    failed = _run_pins(_build(_source(), tmp_path, "original"), tmp_path)
    assert failed == [], failed


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(name, orig, bad, tmp_path):
    src = _source()
    assert src.count(orig) == 1, f"mutation site not found: {orig}"
    failed = _run_pins(_build(src.replace(orig, bad), tmp_path, name), tmp_path)
    assert failed is None or failed, f"{name}: every pin passed"
