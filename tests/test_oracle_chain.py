"""Pins of the oracle's whole rational program (Section IV, steps 4-5).

tests/golden/chain_cases.json holds two hand-made kernels whose metrics are
exact binary fractions, and the cycles, choices, margins and status bits
worked out by hand from the paper's definitions: the metric map with |g|, a
denominator that vanishes at one block shape, #blocks = ceil(N/T),
#active_SMs = min(#SM, #blocks), whole waves #Rep, the non-strict
meaningful test b_i <= N, and a query with no meaningful configuration.

The mutation test plants, one at a time, the mistakes those cases are meant to
catch into a private copy of ``oracle.program`` (on the CPU; the oracle
itself is untouched) and checks that each one breaks at least one case.
"""
import importlib.util
import json
import math
import os
import types

import numpy as np
import pytest

from oracle import configs, program

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chain_cases.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _program(g, name):
    k = g["kernels"][name]
    return dict(coef=np.array(k["coef"], dtype=np.float64)[None], regs=np.array([k["regs"]]),
                smem=np.array([k["smem"]]), n_vars=g["n_vars"], degree=g["degree"],
                n_scale_log2=g["n_scale_log2"], b_scale_log2=g["b_scale_log2"],
                metric_lo=g["metric_lo"], metric_scale=g["metric_scale"])


def _mismatches(prog_mod, g):
    """Every golden expectation that prog_mod (a module with choose and
    evaluate_kernel) does not meet, as readable strings."""
    F = configs.enumerate_configs(2)
    bad = []
    for c in g["queries"]:
        p = _program(g, c["kernel"])
        r = prog_mod.choose(p, g["hw"], F, np.array([0, 1]), np.array([c["N"]], dtype=np.int64))
        tag = f'{c["kernel"]} N={c["N"]}'
        if int(r["best"][0]) != c["best"]:
            bad.append(f"{tag}: best {int(r['best'][0])} != {c['best']}")
            continue
        if c["best"] >= 0 and tuple(F[c["best"]]) != tuple(c["best_config"]):
            bad.append(f"{tag}: index {c['best']} is {F[c['best']]}, not {c['best_config']}")
        if int(r["status"][0]) != c["status"]:
            bad.append(f"{tag}: status {int(r['status'][0])} != {c['status']}")
        if c["best_cycles"] is None:
            if math.isfinite(float(r["best_cycles"][0])):
                bad.append(f"{tag}: cycles {r['best_cycles'][0]} for an infeasible query")
        elif r["best_cycles"][0] != pytest.approx(c["best_cycles"], rel=1e-12):
            bad.append(f"{tag}: cycles {r['best_cycles'][0]} != {c['best_cycles']}")
        if float(r["margin"][0]) != pytest.approx(c["margin"], rel=1e-12, abs=1e-15):
            bad.append(f"{tag}: margin {r['margin'][0]} != {c['margin']}")
    for c in g["cells"]:
        k = g["kernels"][c["kernel"]]
        ev = prog_mod.evaluate_kernel(np.array(k["coef"]), k["regs"], k["smem"], [c["N"]], F,
                                      g["hw"], g["metric_lo"], g["metric_scale"], g["n_vars"],
                                      g["degree"], g["n_scale_log2"], g["b_scale_log2"])
        j = F.index(tuple(c["config"]))
        tag = f'{c["kernel"]} N={c["N"]} b={tuple(c["config"])}'
        if bool(ev["valid"][0, j]) != c["valid"]:
            bad.append(f"{tag}: valid {ev['valid'][0, j]}")
        if bool(ev["meaningful"][0, j]) != c["meaningful"]:
            bad.append(f"{tag}: meaningful {ev['meaningful'][0, j]}")
        got = float(ev["cycles"][0, j])
        if c["cycles"] is None:
            if math.isfinite(got):
                bad.append(f"{tag}: cycles {got} for an unusable configuration")
            continue
        if got != pytest.approx(c["cycles"], rel=1e-12):
            bad.append(f"{tag}: cycles {got} != {c['cycles']}")
        if int(ev["branch"][0, j]) != c["branch"]:
            bad.append(f"{tag}: branch {int(ev['branch'][0, j])} != {c['branch']}")
        if int(ev["n_blocks"][0, j]) != c["n_blocks"] or int(ev["rep"][0, j]) != c["rep"]:
            bad.append(f"{tag}: blocks/rep {int(ev['n_blocks'][0, j])}/{int(ev['rep'][0, j])}")
    return bad


def test_chain_golden_cases():
    g = _golden()
    assert len(g["queries"]) >= 7 and len(g["cells"]) >= 6
    bad = _mismatches(program, g)
    assert not bad, "\n".join(bad)


def test_chain_golden_kernels_are_exact():
    """The hand-made metrics are what the `why` fields say, at every shape."""
    from oracle import rational
    g = _golden()
    F = configs.enumerate_configs(2)
    exps = rational.monomial_exponents(3, 2)
    raw = np.array([(1 << 12, b0, b1) for b0, b1 in F], dtype=np.float64)
    xs = rational.scale_variables(raw, 23, 10)
    L, valid = program.metrics(np.array(g["kernels"]["A"]["coef"]), xs, exps,
                               g["metric_lo"], g["metric_scale"])
    b1 = np.array([b for _, b in F], dtype=np.float64)
    assert np.array_equal(L[0], 100 + b1 / 16)
    assert np.all(L[1] == 10) and np.all(L[6] == 152) and np.all(L[7] == 4)
    assert np.all(L[2] == 0) and np.all(L[3] == 0) and np.all(L[4] == 1)
    bad = [j for j, s in enumerate(F) if not valid[j]]
    assert bad == [F.index((32, 32))]
    LB, vB = program.metrics(np.array(g["kernels"]["B"]["coef"]), xs, exps,
                             g["metric_lo"], g["metric_scale"])
    assert vB.all()
    assert [float(v[0]) for v in LB] == [100, 10, 0, 1, 1, 1, 512, 4]


# (original text in oracle/program.py, planted mistake)
MUTATIONS = [
    ("return lo + sc * np.abs(g), valid", "return lo + sc * g, valid"),
    ("n_blocks = -(-N[:, None] // T[None, :])", "n_blocks = (N[:, None] // T[None, :])"),
    ("rep = -(-n_blocks // per_wave)", "rep = n_blocks / per_wave"),
    ("rep = -(-n_blocks // per_wave)", "rep = np.maximum(n_blocks // per_wave, 1)"),
    ('active_sms = np.minimum(hw["n_sm"], n_blocks)',
     'active_sms = np.full_like(n_blocks, hw["n_sm"])'),
    ("cfg[None, :, :] <= N[:, None, None]", "cfg[None, :, :] < N[:, None, None]"),
    ("valid = np.all((q != 0) & np.isfinite(g), axis=0)",
     "valid = np.all(np.isfinite(q), axis=0)"),
]


@pytest.mark.parametrize("orig,planted", MUTATIONS)
def test_chain_golden_cases_catch_planted_mistakes(orig, planted):
    path = os.path.join(os.path.dirname(program.__file__), "program.py")
    src = open(path).read()
    assert orig in src, f"oracle/program.py no longer contains {orig!r}"
    mod = types.ModuleType("oracle._planted_program")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, planted), path + " (planted)", "exec"), mod.__dict__)
    assert _mismatches(mod, _golden()), f"the chain cases do not notice {planted!r}"
