"""Oracle: hardware occupancy as a rational program (test infrastructure only).

Example 1 and Fig. 1 of the paper: the number of active blocks per SM,
B_active, is decided by a cascade of four tests on the hardware limits
(blocks per SM B_max, warps per SM W_max, registers per SM R_max, shared memory
per SM Z_max) and the kernel's registers per thread R, shared memory per block Z
and threads per block T.  The first test that holds sets B_active; if none holds
the kernel fails to launch (B_active = 0).  Eq. 1 then gives
W_active = min(floor(B_active T / 32), W_max).

Readings (the figure is the authority where the text differs):
* R_max and Z_max are per-SM limits, as the flowchart uses them (Example 1's
  list calls them per-block);
* the unbalanced parenthesis of the register node reads floor(R_max / (R T));
* R = 0 or Z = 0 means the kernel uses none of that resource: the cascade's
  inequalities are evaluated as written, and a test whose formula would divide by
  zero is one that cannot hold;
* T > T_max (listed in Example 1, unused in Fig. 1) also means failure to launch.
All arithmetic is on Python integers.
"""
from __future__ import annotations


def active_blocks(T: int, R: int, Z: int, hw: dict) -> int:
    """B_active by the Fig. 1 cascade, in the figure's order."""
    Bm, Wm = hw["max_blocks_per_sm"], hw["max_warps_per_sm"]
    Rm, Zm = hw["regs_per_sm"], hw["smem_per_sm"]
    if T > hw["max_threads_per_block"] or T <= 0:
        return 0
    # 1. nothing limits: the block-count limit is reached
    if T * Bm <= 32 * Wm and R * T * Bm <= Rm and Z * Bm <= Zm:
        return Bm
    # 2. warps limit
    if 32 * Wm <= T * Bm and 32 * Wm * R <= Rm and 32 * Wm * Z <= Zm * T:
        return (32 * Wm) // T
    # 3. registers limit
    if R > 0 and Rm <= R * T * Bm and Rm <= R * 32 * Wm and Rm * Z <= R * T * Zm:
        return Rm // (R * T)
    # 4. shared memory limits
    if Z > 0 and Zm <= Bm * Z and Zm * T <= 32 * Wm * Z and Zm * R * T <= Z * Rm:
        return Zm // Z
    return 0


def active_warps(B_active: int, T: int, hw: dict) -> int:
    """Eq. 1: W_active = min(floor(B_active T / 32), W_max)."""
    return min((B_active * T) // 32, hw["max_warps_per_sm"])
