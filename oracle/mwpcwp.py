"""Oracle: the MWP-CWP execution-time model (test infrastructure only).

Example 2 of the paper names MWP-CWP (Hong and Kim, ISCA 2009; Sim et al.,
PPoPP 2012) as the high-level model whose execution time KLARAPTOR's rational
program computes from low-level metrics, hardware parameters and the block
size.  The paper does not print the model's equations and its code-generation
section is omitted from the text, so this module restates the published model:

* memory latency of a warp access, coalesced and uncoalesced, from the base
  latency and the departure delay per extra transaction;
* MWP (memory warp parallelism) = min(latency / departure delay,
  bandwidth-limited MWP, active warps N);
* CWP (compute warp parallelism) = min((memory + compute cycles) / compute
  cycles, N);
* three cases: both saturated at N; memory-bound or compute-dominated; and
  latency-bound;
* plus the synchronisation cost departure_delay (MWP - 1) #synch B_active #Rep.

Readings of this project: a coalesced warp access also pays
(coal_per_mw - 1) departure delays (reduces to the published model at
coal_per_mw = 1); #Rep = ceil(#blocks / (B_active #active_SMs)) in whole waves;
#blocks = ceil(N / T) and #active_SMs = min(#SMs, #blocks); N = W_active of
Eq. 1.

Parity unpinned: fidelity to the paper's own generated MWP-CWP code cannot be
checked (that code is not in the paper).  The tests pin this restatement with
hand-worked cases, one per branch.

Works elementwise on numpy arrays (or Python floats).
"""
from __future__ import annotations

import numpy as np


def cycles(L, hw, W_active, B_active, active_sms, rep):
    """Execution cycles by MWP-CWP.

    L: sequence of the eight metric arrays (comp, coal, uncoal, synch,
    coal_per_mw, uncoal_per_mw, load_bytes_per_warp, issue_cycles).
    Returns (cycles, branch (1, 2 or 3), boundary_margin) where boundary_margin
    is the smallest relative distance of a branch decision to its threshold.
    """
    comp, coal, uncoal, synch, coal_mw, uncoal_mw, load_bytes, issue = L
    Nw = np.asarray(W_active, dtype=np.float64)
    Bact = np.asarray(B_active, dtype=np.float64)
    rep = np.asarray(rep, dtype=np.float64)
    active_sms = np.asarray(active_sms, dtype=np.float64)
    mem_ld = hw["mem_latency"]
    dep_c, dep_u = hw["departure_delay_coal"], hw["departure_delay_uncoal"]

    mem_l_uncoal = mem_ld + (uncoal_mw - 1.0) * dep_u
    mem_l_coal = mem_ld + (coal_mw - 1.0) * dep_c
    mem_insts = coal + uncoal
    w_u = uncoal / mem_insts
    w_c = coal / mem_insts
    mem_l = mem_l_uncoal * w_u + mem_l_coal * w_c
    departure = dep_u * uncoal_mw * w_u + dep_c * coal_mw * w_c

    mwp_nobw = mem_l / departure
    bw_per_warp = hw["clock_hz"] * load_bytes / mem_l
    mwp_peakbw = hw["mem_bandwidth"] / (bw_per_warp * active_sms)
    mwp = np.minimum(np.minimum(mwp_nobw, mwp_peakbw), Nw)

    comp_cycles = issue * (comp + coal + uncoal)
    mem_cycles = mem_l_uncoal * uncoal + mem_l_coal * coal
    cwp_full = (mem_cycles + comp_cycles) / comp_cycles
    cwp = np.minimum(cwp_full, Nw)

    c1 = mwp == Nw
    c2 = cwp == Nw
    c3 = cwp >= mwp
    c4 = comp_cycles > mem_cycles
    e1 = (mem_cycles + comp_cycles + comp_cycles / mem_insts * (mwp - 1.0)) * rep
    e2 = (mem_cycles * Nw / mwp + comp_cycles / mem_insts * (mwp - 1.0)) * rep
    e3 = (mem_l + comp_cycles * Nw) * rep
    branch = np.where(c1 & c2, 1, np.where(c3 | c4, 2, 3))
    e = np.where(branch == 1, e1, np.where(branch == 2, e2, e3))
    e = e + departure * (mwp - 1.0) * synch * Bact * rep

    # distance of each decision to its threshold, relative
    m1 = np.abs(np.minimum(mwp_nobw, mwp_peakbw) - Nw) / Nw
    m2 = np.abs(cwp_full - Nw) / Nw
    m3 = np.abs(cwp - mwp) / np.maximum(cwp, mwp)
    m4 = np.abs(comp_cycles - mem_cycles) / np.maximum(comp_cycles, mem_cycles)
    # branch 1 <=> c1 and c2: robust if both hold robustly, or one fails robustly
    d12 = np.where(c1 & c2, np.minimum(m1, m2),
                   np.maximum(np.where(c1, 0.0, m1), np.where(c2, 0.0, m2)))
    # c3 or c4: robust if a true clause holds robustly, or both fail robustly
    d34 = np.where(c3 | c4, np.maximum(np.where(c3, m3, 0.0), np.where(c4, m4, 0.0)),
                   np.minimum(m3, m4))
    margin = np.where(branch == 1, d12, np.minimum(d12, d34))
    return e, branch, margin
