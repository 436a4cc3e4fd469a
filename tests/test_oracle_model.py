"""Pins of the oracle's configuration set, occupancy, MWP-CWP and argmin.

Each test checks the oracle against something other than itself: closed-form
counts, hand-worked cases (tests/golden), brute force over a plain definition,
or invariants that a dropped term, swapped operand or wrong index would break.
A mutation test plants such mistakes one at a time in private copies of the
occupancy and MWP-CWP modules and checks that each breaks at least one pin.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import configs, mwpcwp, occupancy, program

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- configuration set F (Section IV step 4; Section V) ---------------------

def test_config_counts_closed_form():
    # thread counts 2^k, k = 5..10; 2D shapes with product 2^k: k+1; 3D: (k+1)(k+2)/2
    assert len(configs.enumerate_configs(2)) == sum(k + 1 for k in range(5, 11)) == 51
    assert len(configs.enumerate_configs(3)) == sum((k + 1) * (k + 2) // 2
                                                    for k in range(5, 11)) == 251
    assert len(configs.enumerate_configs(1)) == 6


def test_config_constraints_and_order():
    F = configs.enumerate_configs(3)
    T = [math.prod(c) for c in F]
    assert all(t % 32 == 0 and 32 <= t <= 1024 for t in T)
    assert T == sorted(T)
    assert len(set(F)) == len(F)
    assert F[0] == (32, 1, 1) and F[-1] == (1, 1, 1024)
    F2 = configs.enumerate_configs(2)
    assert F2[:3] == [(32, 1), (16, 2), (8, 4)]
    # brute force over all power-of-two shapes up to 1024 per dimension
    brute = [s for s in itertools.product([1 << e for e in range(11)], repeat=2)
             if 32 <= s[0] * s[1] <= 1024]
    assert sorted(brute) == sorted(F2)


# --- occupancy (Fig. 1, Eq. 1) ------------------------------------------------

def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_occupancy_hand_cases():
    g = _golden("occupancy_cases.json")
    for c in g["cases"]:
        B = occupancy.active_blocks(c["T"], c["R"], c["Z"], g["hw"])
        assert B == c["B_active"], c
        assert occupancy.active_warps(B, c["T"], g["hw"]) == c["W_active"], c


HW = dict(max_blocks_per_sm=32, max_warps_per_sm=64, regs_per_sm=65536,
          smem_per_sm=233472, max_threads_per_block=1024)


def _floor_of_min(T, R, Z, hw):
    """The plain definition the cascade computes: floor of the tightest limit."""
    lims = [hw["max_blocks_per_sm"], (32 * hw["max_warps_per_sm"]) // T]
    if R:
        lims.append(hw["regs_per_sm"] // (R * T))
    if Z:
        lims.append(hw["smem_per_sm"] // Z)
    return min(lims)


def test_occupancy_cascade_is_floor_of_min_bruteforce():
    Ts = list(range(32, 1025, 32))
    Zs = list(range(0, 233473, 4096)) + [233472, 233473]
    for T in Ts:
        for R in range(0, 256, 3):
            for Z in Zs:
                assert occupancy.active_blocks(T, R, Z, HW) == _floor_of_min(T, R, Z, HW), (T, R, Z)


def test_occupancy_invariants():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        T = int(rng.choice([32, 64, 128, 256, 512, 1024, 96, 160]))
        R = int(rng.integers(1, 256))
        Z = int(rng.integers(0, 233473))
        B = occupancy.active_blocks(T, R, Z, HW)
        W = occupancy.active_warps(B, T, HW)
        assert B * R * T <= HW["regs_per_sm"]
        assert B * Z <= HW["smem_per_sm"]
        assert B * T <= 32 * HW["max_warps_per_sm"]
        assert 0 <= W <= HW["max_warps_per_sm"]
        # monotone non-increasing in R and Z
        assert occupancy.active_blocks(T, R + 1, Z, HW) <= B
        assert occupancy.active_blocks(T, R, Z + 1024, HW) <= B


# --- MWP-CWP (Example 2) -----------------------------------------------------

def test_mwpcwp_hand_cases():
    g = _golden("mwpcwp_cases.json")
    for c in g["cases"]:
        e, br, _ = mwpcwp.cycles([np.float64(v) for v in c["L"]], g["hw"], c["W_active"],
                                 c["B_active"], c["active_sms"], c["rep"])
        assert int(br) == c["branch"], c["name"]
        assert float(e) == pytest.approx(c["cycles"], rel=1e-12), c["name"]


def test_mwpcwp_synch_term_vanishes_at_mwp_one():
    hw = dict(mem_latency=600.0, departure_delay_coal=4.0, departure_delay_uncoal=10.0,
              mem_bandwidth=8.0e12, clock_hz=1.9e9)
    L = [np.float64(v) for v in (100, 10, 0, 0, 1, 1, 128, 4)]
    Ls = list(L)
    Ls[3] = np.float64(50)
    a, _, _ = mwpcwp.cycles(L, hw, 1, 1, 148, 1)      # N = 1 forces MWP = 1
    b, _, _ = mwpcwp.cycles(Ls, hw, 1, 1, 148, 1)
    assert float(a) == float(b)
    # and it is linear in the synch count when MWP > 1
    c1, _, _ = mwpcwp.cycles(Ls, hw, 8, 2, 148, 1)
    Ls[3] = np.float64(100)
    c2, _, _ = mwpcwp.cycles(Ls, hw, 8, 2, 148, 1)
    c0, _, _ = mwpcwp.cycles(L, hw, 8, 2, 148, 1)
    assert float(c2 - c0) == pytest.approx(2 * float(c1 - c0), rel=1e-12)


def test_mwpcwp_linear_in_rep():
    hw = dict(mem_latency=600.0, departure_delay_coal=4.0, departure_delay_uncoal=10.0,
              mem_bandwidth=8.0e12, clock_hz=1.9e9)
    rng = np.random.default_rng(3)
    for _ in range(200):
        L = [rng.uniform(1, 500), rng.uniform(1, 30), rng.uniform(0, 8), rng.uniform(0, 4),
             rng.uniform(1, 5), rng.uniform(1, 32), rng.uniform(32, 512), rng.uniform(1, 9)]
        L = [np.float64(v) for v in L]
        W = int(rng.integers(1, 65))
        e1, b1, _ = mwpcwp.cycles(L, hw, W, 2, 148, 1)
        e5, b5, _ = mwpcwp.cycles(L, hw, W, 2, 148, 5)
        assert b1 == b5
        assert float(e5) == pytest.approx(5 * float(e1), rel=1e-12)
        assert float(e1) > 0


# --- argmin (Section IV step 5) ------------------------------------------------

def _brute_argmin(row):
    best, val = -1, math.inf
    for i, v in enumerate(row):
        if math.isfinite(v) and v < val:
            best, val = i, v
    return best, val


def test_argmin_bruteforce_and_ties():
    rng = np.random.default_rng(1)
    for _ in range(500):
        n = int(rng.integers(1, 12))
        row = rng.integers(0, 6, n).astype(np.float64)   # many exact ties
        row[rng.random(n) < 0.2] = np.inf
        b, v, mg = program.argmin(row[None, :])
        eb, ev = _brute_argmin(row)
        assert b[0] == eb
        if eb >= 0:
            assert v[0] == ev
            rest = [x for j, x in enumerate(row) if j != eb and math.isfinite(x)]
            want = (min(rest) - ev) / ev if rest else math.inf
            if ev == 0:
                continue
            assert mg[0] == pytest.approx(want) if math.isfinite(want) else mg[0] == math.inf


def test_argmin_permutation_invariance():
    rng = np.random.default_rng(2)
    for _ in range(200):
        row = rng.uniform(1, 2, 20)
        perm = rng.permutation(20)
        b, v, _ = program.argmin(row[None, :])
        bp, vp, _ = program.argmin(row[perm][None, :])
        assert v[0] == vp[0] and perm[bp[0]] == b[0]


def test_launch_params():
    assert program.launch_params((32, 8), 1000) == (32, 125, 1, 32, 8, 1)
    assert program.launch_params((4, 4, 2), 9) == (3, 3, 5, 4, 4, 2)


def test_refine_reduces_to_argmin_and_prefers_occupancy():
    from oracle import program as P
    rng = np.random.default_rng(11)
    cyc = rng.uniform(100, 200, (40, 12))
    cyc[rng.random((40, 12)) < 0.2] = np.inf
    cyc[5, :] = np.inf
    W = rng.integers(1, 64, 12)
    # eps = 0: the plain argmin (lowest index among equal values)
    cyc[7, 3] = cyc[7, 9] = cyc[7][np.isfinite(cyc[7])].min() - 1.0
    b0 = P.refine(cyc, W, 0.0)
    want, _, _ = P.argmin(cyc)
    # with eps = 0 equal values can still differ in warps: only exact ties move
    exact = np.array([np.sum(cyc[r] == cyc[r][np.isfinite(cyc[r])].min()) == 1 if np.isfinite(cyc[r]).any()
                      else True for r in range(40)])
    assert np.array_equal(b0[exact], want[exact])
    assert b0[5] == -1
    # brute force for a larger margin
    eps = 0.1
    b = P.refine(cyc, W, eps)
    for r in range(40):
        fin = np.isfinite(cyc[r])
        if not fin.any():
            continue
        lo = cyc[r][fin].min()
        cand = [c for c in range(12) if fin[c] and cyc[r, c] <= lo * (1 + eps)]
        wmax = max(W[c] for c in cand)
        assert W[b[r]] == wmax and b[r] in cand
        assert cyc[r, b[r]] == min(cyc[r, c] for c in cand if W[c] == wmax)
    # a wider margin never lowers the occupancy of the choice
    for e1, e2 in ((0.0, 0.05), (0.05, 0.2), (0.2, 1.0)):
        b1, b2 = P.refine(cyc, W, e1), P.refine(cyc, W, e2)
        ok = b1 >= 0
        assert np.all(W[b2[ok]] >= W[b1[ok]])


# --- planted mistakes ------------------------------------------------------------
# The occupancy and MWP-CWP pins above, run against private copies of the
# oracle modules with one plausible mistake planted at a time (on the CPU; the
# oracle itself is untouched): each mistake must break at least one pin.

def _planted_module(module, orig, planted):
    import types
    path = module.__file__
    src = open(path).read()
    assert src.count(orig) == 1, f"{os.path.basename(path)} no longer holds {orig!r} once"
    mod = types.ModuleType("oracle._planted_" + module.__name__.rsplit(".", 1)[-1])
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, planted), path + " (planted)", "exec"), mod.__dict__)
    return mod


def _fails(fn):
    try:
        fn()
    except Exception:  # an assertion or a crash: the pin noticed
        return True
    return False


def _occupancy_pin_failures(occ):
    def hand():
        g = _golden("occupancy_cases.json")
        for c in g["cases"]:
            B = occ.active_blocks(c["T"], c["R"], c["Z"], g["hw"])
            assert B == c["B_active"] and occ.active_warps(B, c["T"], g["hw"]) == c["W_active"]

    def brute():
        for T in range(32, 1025, 32):
            for R in range(0, 256, 9):
                for Z in list(range(0, 233473, 16384)) + [233472, 233473]:
                    assert occ.active_blocks(T, R, Z, HW) == _floor_of_min(T, R, Z, HW)

    def bounds():
        rng = np.random.default_rng(0)
        for _ in range(500):
            T = int(rng.choice([32, 64, 128, 256, 512, 1024, 96, 160]))
            R, Z = int(rng.integers(1, 256)), int(rng.integers(0, 233473))
            B = occ.active_blocks(T, R, Z, HW)
            W = occ.active_warps(B, T, HW)
            assert B * R * T <= HW["regs_per_sm"] and B * Z <= HW["smem_per_sm"]
            assert B * T <= 32 * HW["max_warps_per_sm"] and 0 <= W <= HW["max_warps_per_sm"]
            assert W == min(B * T // 32, HW["max_warps_per_sm"])

    return [n for n, fn in (("hand", hand), ("brute", brute), ("bounds", bounds)) if _fails(fn)]


def _mwpcwp_pin_failures(mc):
    hw = dict(mem_latency=600.0, departure_delay_coal=4.0, departure_delay_uncoal=10.0,
              mem_bandwidth=8.0e12, clock_hz=1.9e9)

    def hand():
        g = _golden("mwpcwp_cases.json")
        for c in g["cases"]:
            e, br, _ = mc.cycles([np.float64(v) for v in c["L"]], g["hw"], c["W_active"],
                                 c["B_active"], c["active_sms"], c["rep"])
            assert int(br) == c["branch"] and float(e) == pytest.approx(c["cycles"], rel=1e-12)

    def synch():
        L = [np.float64(v) for v in (100, 10, 0, 0, 1, 1, 128, 4)]
        Ls = list(L)
        Ls[3] = np.float64(50)
        assert float(mc.cycles(L, hw, 1, 1, 148, 1)[0]) == float(mc.cycles(Ls, hw, 1, 1, 148, 1)[0])
        c0 = float(mc.cycles(L, hw, 8, 2, 148, 1)[0])
        c1 = float(mc.cycles(Ls, hw, 8, 2, 148, 1)[0])
        Ls[3] = np.float64(100)
        c2 = float(mc.cycles(Ls, hw, 8, 2, 148, 1)[0])
        assert c2 - c0 == pytest.approx(2 * (c1 - c0), rel=1e-12)

    def rep():
        rng = np.random.default_rng(3)
        for _ in range(200):
            L = [np.float64(v) for v in (
                rng.uniform(1, 500), rng.uniform(1, 30), rng.uniform(0, 8), rng.uniform(0, 4),
                rng.uniform(1, 5), rng.uniform(1, 32), rng.uniform(32, 512), rng.uniform(1, 9))]
            W = int(rng.integers(1, 65))
            e1, b1, _ = mc.cycles(L, hw, W, 2, 148, 1)
            e5, b5, _ = mc.cycles(L, hw, W, 2, 148, 5)
            assert b1 == b5 and float(e5) == pytest.approx(5 * float(e1), rel=1e-12)
            assert float(e1) > 0

    return [n for n, fn in (("hand", hand), ("synch", synch), ("rep", rep)) if _fails(fn)]


# (original text, planted mistake)
OCCUPANCY_MUTATIONS = [
    ("if T * Bm <= 32 * Wm and R * T * Bm <= Rm and Z * Bm <= Zm:",
     "if T * Bm <= 32 * Wm and R * Bm <= Rm and Z * Bm <= Zm:"),
    ("return (32 * Wm) // T", "return Wm // T"),
    ("return Rm // (R * T)", "return Rm // R"),
    ("return Zm // Z", "return Zm // (Z * T)"),
    ('return min((B_active * T) // 32, hw["max_warps_per_sm"])',
     'return max((B_active * T) // 32, hw["max_warps_per_sm"])'),
    ('if T > hw["max_threads_per_block"] or T <= 0:',
     'if T >= hw["max_threads_per_block"] or T <= 0:'),
]
MWPCWP_MUTATIONS = [
    ("mem_l_uncoal = mem_ld + (uncoal_mw - 1.0) * dep_u",
     "mem_l_uncoal = mem_ld + uncoal_mw * dep_u"),
    ("mem_l = mem_l_uncoal * w_u + mem_l_coal * w_c",
     "mem_l = mem_l_uncoal * w_c + mem_l_coal * w_u"),
    ("departure = dep_u * uncoal_mw * w_u + dep_c * coal_mw * w_c",
     "departure = dep_u * w_u + dep_c * w_c"),
    ("mwp = np.minimum(np.minimum(mwp_nobw, mwp_peakbw), Nw)",
     "mwp = np.minimum(mwp_nobw, Nw)"),
    ('mwp_peakbw = hw["mem_bandwidth"] / (bw_per_warp * active_sms)',
     'mwp_peakbw = hw["mem_bandwidth"] / bw_per_warp'),
    ("comp_cycles = issue * (comp + coal + uncoal)", "comp_cycles = issue * comp"),
    ("cwp = np.minimum(cwp_full, Nw)", "cwp = cwp_full"),
    ("c4 = comp_cycles > mem_cycles", "c4 = comp_cycles < mem_cycles"),
    ("branch = np.where(c1 & c2, 1, np.where(c3 | c4, 2, 3))",
     "branch = np.where(c1 | c2, 1, np.where(c3 | c4, 2, 3))"),
    ("e1 = (mem_cycles + comp_cycles + comp_cycles / mem_insts * (mwp - 1.0)) * rep",
     "e1 = (mem_cycles + comp_cycles + comp_cycles / mem_insts * (mwp + 1.0)) * rep"),
    ("e2 = (mem_cycles * Nw / mwp + comp_cycles / mem_insts * (mwp - 1.0)) * rep",
     "e2 = (mem_cycles * mwp / Nw + comp_cycles / mem_insts * (mwp - 1.0)) * rep"),
    ("e3 = (mem_l + comp_cycles * Nw) * rep", "e3 = (mem_l + comp_cycles) * rep"),
    ("e = e + departure * (mwp - 1.0) * synch * Bact * rep",
     "e = e + departure * (mwp - 1.0) * synch * Bact"),
]


def test_model_pins_pass_on_the_oracle():
    assert _occupancy_pin_failures(occupancy) == []
    assert _mwpcwp_pin_failures(mwpcwp) == []


@pytest.mark.parametrize("orig,planted", OCCUPANCY_MUTATIONS)
def test_occupancy_pins_catch_planted_mistakes(orig, planted):
    assert _occupancy_pin_failures(_planted_module(occupancy, orig, planted)), planted


@pytest.mark.parametrize("orig,planted", MWPCWP_MUTATIONS)
def test_mwpcwp_pins_catch_planted_mistakes(orig, planted):
    assert _mwpcwp_pin_failures(_planted_module(mwpcwp, orig, planted)), planted
