"""Two-site sweeps (Sec. 2.1) on the GPU against the FP64 oracle DMRG, step by step.

Both sides run the same schedule from the Aufbau product state (forward over
positions 0..L-3, backward over L-2..1; at each step the lowest eigenpair of
Eq. h_mat, then the truncation to M states and the renormalization of
Eq. renorm_mat), so every step's energy must agree to 1e-10 Eh.  Both cut the
density-matrix spectrum below a near-degenerate cluster that straddles the M-th
eigenvalue, so the kept space does not depend on rounding.  The one exception
is a top cluster larger than M, which cannot be cut that way (a gap below 1e-10
left at the cut, reported by dmrg_truncation_stats): the two codes may then
keep different but equally valid states, and that step and the later ones are
compared at 1e-8 Eh.

Further invariants: every energy is a variational upper bound of the full-CI
energy (where FCI is affordable), and the lowest energy of a sweep does not
rise over sweeps by more than the truncation can explain.
"""
import os

import numpy as np
import pytest

from oracle import dmrg as od
from oracle import fock
from paper_2001_04890_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def stepped_sweeps(ctx, nsw, tol, max_iter=300):
    """The dmrg_sweep schedule, one step at a time: per step (energy, discarded
    weight, straddled cut at this step)."""
    L = ctx.L
    ctx.set_position(0, 1)
    out = []
    for _ in range(nsw):
        for direction, ks in ((+1, range(0, L - 2)), (-1, range(L - 2, 0, -1))):
            for _k in ks:
                e, _ = ctx.davidson(tol=tol, max_iter=max_iter, allow_noconv=True)
                dw, _ = ctx.renormalize(direction)
                st = ctx.truncation_stats()
                out.append((e, dw, st["last_gap"] < 1e-10))
    E = np.array([o[0] for o in out])
    DW = np.array([o[1] for o in out])
    S = np.array([o[2] for o in out])
    return E, DW, S


def assert_steps_match(E, ref, straddled):
    """1e-10 Eh per step; 1e-8 Eh from the first straddled cut on."""
    first = int(np.argmax(straddled)) if straddled.any() else len(E)
    tol = np.where(np.arange(len(E)) < first, 1e-10, 1e-8)
    bad = np.nonzero(np.abs(E - ref) > tol)[0]
    assert bad.size == 0, (bad[:5], (E - ref)[bad[:5]], first)


def assert_sweep_minima_monotone(E, DW, nsw):
    """Lowest energy per sweep non-increasing, within what the truncation can move it."""
    Es, Ds = E.reshape(nsw, -1), DW.reshape(nsw, -1)
    mins = Es.min(axis=1)
    for s in range(1, nsw):
        slack = 1e-10 + 10.0 * Ds[s].max() * abs(mins[s])
        assert mins[s] <= mins[s - 1] + slack, (s, mins)


def read_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_l8_m64_sweeps_match_oracle():
    """L=8, N=8, Sz=0, M=64, six sweeps: every step equals the oracle's (1e-10 Eh)."""
    L, N, M, nsw = 8, 8, 64, 6
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    E, DW, S = stepped_sweeps(ctx, nsw, tol=1e-10)
    ctx.close()
    ref = od.OracleDMRG(h, v, N, 0, M).sweep(nsw, tol=1e-10)
    assert_steps_match(E, ref, S)
    e_fci = fock.fci_ground(h, v, 4, 4)[0]
    assert np.all(E >= e_fci - 1e-10) and np.all(ref >= e_fci - 1e-10)
    assert_sweep_minima_monotone(E, DW, nsw)


def test_sweep_api_equals_stepped_schedule():
    """dmrg_sweep runs the same steps as the stepped schedule above (same energies)."""
    L, N, M, nsw = 8, 8, 64, 2
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, N, 0, M)
    E1 = ctx.sweep(nsw, tol=1e-10)
    ctx.close()
    ctx = binding.DMRG(h, v, N, 0, M)
    E2, _, _ = stepped_sweeps(ctx, nsw, tol=1e-10)
    ctx.close()
    assert np.max(np.abs(E1 - E2)) < 1e-11


@pytest.mark.parametrize("L,M,nsw", [(12, 128, 4), (24, 32, 2)])
def test_sweeps_match_stored_oracle_energies(L, M, nsw):
    """Per-step energies equal the oracle's stored ones (tests/golden, written by
    make_oracle_sweeps.py from oracle/ alone)."""
    ref = read_golden(f"oracle_sweeps_L{L}_N{L}_2Sz0_M{M}_S{nsw}.txt")
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, L, 0, M)
    # eigen-tolerance 1e-11 on both sides: a state converged to a residual r differs from
    # the exact one by ~r / gap, which the next truncations carry into later energies
    E, DW, S = stepped_sweeps(ctx, nsw, tol=1e-11)
    ctx.close()
    assert len(E) == len(ref)
    assert_steps_match(E, ref, S)
    assert_sweep_minima_monotone(E, DW, nsw)


@pytest.mark.parametrize("prec", [binding.PREC_FP32, binding.PREC_BF16X3])
def test_mixed_precision_sweeps_match_stored_oracle_energies(prec):
    """The mixed modes (FP32 operator copies, or every block on the tensor cores in
    split-BF16 x3, for the Davidson matvecs; FP64 refinement, truncation and
    renormalization) follow the FP64 oracle's sweeps within the 1e-6 Eh the mixed
    modes promise, step by step."""
    L, M, nsw = 12, 128, 4
    ref = read_golden(f"oracle_sweeps_L{L}_N{L}_2Sz0_M{M}_S{nsw}.txt")
    h, v = workloads.integrals(L, seed=0)
    ctx = binding.DMRG(h, v, L, 0, M, precision=prec)
    if prec == binding.PREC_BF16X3:
        ctx.set_tune(tc_min=1)
    E, DW, _ = stepped_sweeps(ctx, nsw, tol=1e-11)
    ctx.close()
    assert len(E) == len(ref)
    assert np.max(np.abs(E - ref)) < 1e-6, np.max(np.abs(E - ref))
    assert_sweep_minima_monotone(E, DW, nsw)


def test_predicted_psi_is_the_converged_state_once_exact():
    """White's prediction (Sec. 2.1 sweep, psi carried through O): once the sweeps
    have reached the full-CI state (every step at the FCI energy), the state
    predicted for the next position is the converged state there (overlap
    1 - 1e-10), so the next Davidson starts converged."""
    L, N, M = 6, 6, 4096
    h, v = workloads.integrals(L, seed=3)
    e_fci = fock.fci_ground(h, v, 3, 3)[0]
    ctx = binding.DMRG(h, v, N, 0, M)
    E = ctx.sweep(4, tol=1e-11)
    assert np.all(np.abs(E[-2 * (L - 2):] - e_fci) < 1e-10)  # the last sweep is exact
    ctx.set_position(0, 1)
    for k in range(0, L - 3):
        e, _ = ctx.davidson(tol=1e-11, max_iter=300)
        assert abs(e - e_fci) < 1e-10
        ctx.renormalize(+1)
        pred = ctx.get_psi()
        pred /= np.linalg.norm(pred)
        ctx.davidson(tol=1e-11, max_iter=300)
        conv = ctx.get_psi()
        conv /= np.linalg.norm(conv)
        assert abs(abs(pred @ conv) - 1.0) < 1e-10, k
    ctx.close()
