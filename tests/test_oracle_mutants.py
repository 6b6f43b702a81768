"""The oracle pins have teeth: each plants one plausible mistake in a copy of
an oracle's C source (a wrong constant, a dropped or duplicated term, a
wrong sign, index, half or bound, transposed operands, a wrong rounding
rule, a lost carry), builds the copy the way the oracle is built, and runs
that oracle's pins from test_oracle_pins.py against it: at least one pin
must reject every mutant.  The unmutated source, built the same way, must
pass them all, so a rejection is the mistake's doing and not the harness's.
The oracle sources themselves are never changed; the copies live in pytest's
temporary directory."""
import os
import subprocess

import pytest

import test_oracle_pins as P
from oracle import build as ob

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# the pins of each oracle, as (pin, extra keyword arguments)
PINS = {
    "axpy_sum": [(P.test_axpy_closed_form, {}), (P.test_axpy_random_matches_elementwise_definition, {})],
    "exact_sum": [(P.test_exact_sum_matches_fsum_with_cancellation, {"seed": 1}),
                  (P.test_exact_sum_hand_cases, {})],
    "jacobi": [(P.test_jacobi_eigenmode_decay, {"abc": abc}) for abc in [(1, 1, 1), (1, 2, 3), (3, 1, 2)]] +
              [(P.test_jacobi_single_spike, {}), (P.test_jacobi_spike_next_to_boundary, {}),
               (P.test_jacobi_boundary_zero_and_random_grid, {})],
    "stress": [(P.test_stress_oracle_against_memory_model, {})],
    "loops": [(P.test_loops_oracle_elementwise_and_untouched, {})],
    "loops_rpc": [(P.test_loops_rpc_oracle_lines_and_values, {})],
    "synth": [(P.test_synth_oracle_hand_cases, {}), (P.test_synth_oracle_rpc_count, {}),
              (P.test_synth_oracle_fused_multiply_add_rounds_once, {}),
              (P.test_synth_oracle_divergent_iterations, {})],
    "spmv_serve": [(P.test_spmv_serve_oracle_hand_case, {"monkeypatch": None})],
}

# (oracle, text in its source (exactly once), replacement, the mistake)
MUTANTS = [
    ("axpy_sum", "y[i] = 2.5 * x[i] + y[i];", "y[i] = 2.5 * y[i] + x[i];", "operands transposed"),
    ("axpy_sum", "if (i % 1024 == 0)", "if (i % 1024 == 1)", "printed iterations off by one"),
    ("axpy_sum", "s += y[i];", "s += x[i];", "sum of the wrong array"),
    ("exact_sum", "if (rnd && (sticky || (mant & 1)))", "if (rnd)", "ties rounded away, not to even"),
    ("exact_sum", "int p = e - 53 + 1074;", "int p = e - 52 + 1074;", "exponent off by one"),
    ("exact_sum", "int64_t sign = x < 0 ? -1 : 1;", "int64_t sign = 1;", "sign dropped"),
    ("exact_sum", "b >= 0 && !sticky;", "b >= 0 && b > shift - 12 && !sticky;", "sticky bit from the top bits only"),
    ("exact_sum", "m >>= -p;", "m >>= -p + 1;", "subnormal shift off by one"),
    ("exact_sum", "a->d[k + 1] += carry;", "a->d[k + 1] += 0 * carry;", "carry lost"),
    ("jacobi", "v = v / 6.0;", "v = v / 7.0;", "wrong divisor"),
    ("jacobi", "v = v + u[c + sk];", "v = v + u[c + sj];", "a neighbour taken twice, one dropped"),
    ("jacobi", "                    v = v + u[c - sk];\n", "", "a neighbour dropped"),
    ("jacobi", "fabs(v - u[c])", "fabs(v + u[c])", "residual sign"),
    ("jacobi", "i == n - 1 ||", "i == n - 2 ||", "boundary off by one"),
    ("jacobi", "if (d > res)", "if (d < res)", "max taken as min"),
    ("jacobi", 'printf("%d %.17g\\n", s, res);', 'printf("%d %.17g\\n", s - 1, res);', "sweep numbered from 0"),
    ("stress", "p[w / 2] = h ^ 0x5555555555555555ull;", "p[w / 2] = h ^ 0x5555555555555554ull;",
     "wrong middle tag"),
    # (dropping the iteration term (8t + j) would change nothing: the eight
    # consecutive values of one t XOR to 0, so no pin can see it)
    ("stress", "c ^= p[0] ^ p[w / 2] ^ p[w - 1]", "c ^= p[0] ^ p[w / 2]", "a tag read dropped"),
    ("stress", "mix((uint64_t)(8 * t + j + 1))", "mix((uint64_t)(8 * t + j))", "tag index off by one"),
    ("stress", "p[w - 1] = ~h;", "p[w - 2] = ~h;", "last word off by one"),
    ("stress", 'printf("%lld %.6e\\n", (long long)t', 'printf("%lld %.5e\\n", (long long)t', "wrong precision"),
    ("stress", "(double)(h & 0xffff) / 7.0", "(double)(h & 0xfff) / 7.0", "wrong mask"),
    ("loops", "a[k] * x[off[k] + i] + y[off[k] + i]", "a[k] * y[off[k] + i] + x[off[k] + i]",
     "operands transposed"),
    ("loops", "for (int64_t i = 0; i < trips[k]; i++)", "for (int64_t i = 1; i < trips[k]; i++)",
     "first iteration dropped"),
    ("loops_rpc", "if (i % 4096 == 0)", "if (i % 4096 == 1)", "printed iterations off by one"),
    ("loops_rpc", "                v = w[0];", "                v = w[words - 1];", "the wrong heap word read back"),
    ("loops_rpc", "double v = a[k] * x[off[k] + i] + y[off[k] + i];",
     "double v = a[k] * x[off[k] + i] - y[off[k] + i];", "sign of a term"),
    ("synth", "v = fmaf(v, 1.0001f, 0.5f);", "v = v * 1.0001f + 0.5f;", "unfused multiply-add"),
    ("synth", "acc = acc + (float)x[(size_t)k * trip + i];", "acc = acc + (float)x[(size_t)i * nwords + k];",
     "input layout transposed"),
    ("synth", "if ((uint32_t)h < div_t)", "if ((uint32_t)(h >> 32) < div_t)", "divergence from the wrong half"),
    ("synth", "mix(seed + (uint64_t)i * 0x9E3779B97F4A7C15ull)", "mix(seed + (uint64_t)i)", "counter step dropped"),
    ("spmv_serve", "s = s + val[j] * x[col[j]];", "s = s + val[j] * x[i];", "gather index"),
    ("spmv_serve", "        double *t = x;\n        x = y;\n        y = t;\n", "", "passes not chained"),
    ("spmv_serve", "} else if (kind == 1) {", "} else if (kind == 3) {", "request kinds swapped"),
    ("spmv_serve", "((uint64_t)prog << 40)", "((uint64_t)prog << 41)", "record key"),
    ("spmv_serve", '"GF_SERVE_VAR%d", (int)(i % 3)', '"GF_SERVE_VAR%d", (int)(i % 2)', "variable name index"),
]


def _build(name, text, out_dir):
    src = out_dir / (name + ".c")
    src.write_text(text)
    exe = out_dir / name
    subprocess.run(["gcc", *ob.CFLAGS, "-o", str(exe), str(src), "-lm"], check=True, capture_output=True)
    return str(exe)


def _failing_pins(name, exe, tmp_path, monkeypatch):
    """Names of the pins of oracle `name` that reject the binary `exe`."""
    def lookup(n):
        return exe if n == name else ob.binary(n)
    failed = []
    for k, (pin, kw) in enumerate(PINS[name]):
        d = tmp_path / f"pin{k}"
        d.mkdir()
        args = {a: (monkeypatch if a == "monkeypatch" else v) for a, v in kw.items()}
        try:
            pin(lookup, d, **args)
        except Exception:                 # a failed assertion, or a run that exited non-zero
            failed.append(pin.__name__)
    return failed


def test_unmutated_sources_pass_their_pins(oracle_bin, tmp_path, monkeypatch):
    for name in PINS:
        with open(os.path.join(ORACLE, name + ".c")) as f:
            text = f.read()
        d = tmp_path / name
        d.mkdir()
        exe = _build(name, text, d)
        assert _failing_pins(name, exe, d, monkeypatch) == [], name


@pytest.mark.parametrize("name,old,new,what", MUTANTS, ids=[f"{m[0]}-{m[3].replace(' ', '_')}" for m in MUTANTS])
def test_mutant_is_rejected(oracle_bin, tmp_path, monkeypatch, name, old, new, what):
    with open(os.path.join(ORACLE, name + ".c")) as f:
        text = f.read()
    assert text.count(old) == 1, f"{name}: the text to mutate is not there exactly once"
    exe = _build(name, text.replace(old, new), tmp_path)
    assert _failing_pins(name, exe, tmp_path, monkeypatch), f"{name}: no pin rejects the mistake: {what}"
