"""The cyclic-reduction schedules of the coarse block-tridiagonal system (the
library's opt-in elimination order for the exact coarse solve of Section 3.2),
read from the library on the host (ras_coarse_cr_schedule, no CUDA call) and
executed here with dense numpy blocks: for every block count from 1 to 33 the
factorisation and solve schedules solve random block-tridiagonal systems to
rounding, and within a phase no two tasks write one slot or vector and no task
reads what another task of its phase writes (the phases run as parallel work on
the GPU)."""
import os

import numpy as np
import pytest

XV = 1 << 16


@pytest.fixture(scope="module")
def ras():
    from paper_2007_13966_gb300 import build_lib, ras as R
    if not os.path.exists(R.LIB_PATH):
        build_lib.build()
    R.lib()
    return R


def _fac_rounds(fac):
    """[(E, [phase tasks, phase tasks])], last"""
    nround, last, pos, rounds = fac[0], fac[1], 2, []
    for _ in range(nround):
        nE = fac[pos]
        E = fac[pos + 1:pos + 1 + nE]
        pos += 1 + nE
        phases = []
        for _ in range(2):
            n = fac[pos]
            phases.append([fac[pos + 1 + 8 * q:pos + 9 + 8 * q] for q in range(n)])
            pos += 1 + 8 * n
        rounds.append((E, phases))
    assert pos == len(fac)
    return rounds, last


def _sol_phases(sol):
    nph, pos, phases = sol[0], 1, []
    for _ in range(nph):
        n = sol[pos]
        phases.append([sol[pos + 1 + 8 * q:pos + 9 + 8 * q] for q in range(n)])
        pos += 1 + 8 * n
    assert pos == len(sol)
    return phases


def _system(nb, T, rng):
    D = [rng.uniform(-1, 1, (T, T)) + 8 * np.eye(T) for _ in range(nb)]
    Lo = [rng.uniform(-1, 1, (T, T)) if k > 0 else np.zeros((T, T)) for k in range(nb)]
    Up = [rng.uniform(-1, 1, (T, T)) if k + 1 < nb else np.zeros((T, T)) for k in range(nb)]
    A = np.zeros((nb * T, nb * T))
    for k in range(nb):
        A[k * T:(k + 1) * T, k * T:(k + 1) * T] = D[k]
        if k > 0:
            A[k * T:(k + 1) * T, (k - 1) * T:k * T] = Lo[k]
        if k + 1 < nb:
            A[k * T:(k + 1) * T, (k + 1) * T:(k + 2) * T] = Up[k]
    return D, Lo, Up, A


@pytest.mark.parametrize("nb", range(1, 34))
def test_schedule_solves_block_tridiagonal_systems(ras, nb):
    fac, sol, nslot = ras.coarse_cr_schedule(nb)
    rounds, last = _fac_rounds(fac)
    phases = _sol_phases(sol)
    T = 3
    rng = np.random.default_rng(nb)
    D, Lo, Up, A = _system(nb, T, rng)
    S = [None] * (nb + nslot)
    for k in range(nb):
        S[k] = D[k].copy()
        if nslot >= 2 * nb:
            S[nb + k], S[2 * nb + k] = Lo[k].copy(), Up[k].copy()
    for E, fphases in rounds:
        for e in E:
            S[e] = np.linalg.inv(S[e])
        for tasks in fphases:
            new = []
            for out, acc, sign, a1, b1, a2, b2, _ in tasks:
                pr = S[a1] @ S[b1] + (S[a2] @ S[b2] if a2 >= 0 else 0.0)
                new.append((out, (S[out] if acc else 0.0) + sign * pr))
            for out, v in new:
                S[out] = v
    S[last] = np.linalg.inv(S[last])
    b = rng.uniform(-1, 1, nb * T)
    g, x = b.reshape(nb, T).copy(), np.zeros((nb, T))

    def vec(v):
        return (x if v & XV else g)[v & 0xFFFF]

    for tasks in phases:
        new = []
        for out, _, sub, m1, v1, m2, v2, _ in tasks:
            t = S[m1] @ vec(v1) + (S[m2] @ vec(v2) if m2 >= 0 else 0.0)
            new.append((out, vec(out) - t if sub else t))
        for out, v in new:
            (x if out & XV else g)[out & 0xFFFF] = v
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x.ravel() - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("nb", range(3, 65))
def test_phases_are_free_of_hazards(ras, nb):
    fac, sol, _ = ras.coarse_cr_schedule(nb)
    rounds, last = _fac_rounds(fac)
    for E, fphases in rounds:
        assert len(set(E)) == len(E)
        for tasks in fphases:
            writes = [t[0] for t in tasks]
            assert len(set(writes)) == len(writes)
            reads = {r for t in tasks for r in (t[3], t[4]) + ((t[5], t[6]) if t[5] >= 0 else ())}
            assert not reads & set(writes)
    for tasks in _sol_phases(sol):
        writes = [t[0] for t in tasks]
        assert len(set(writes)) == len(writes)
        reads = {t[4] for t in tasks} | {t[6] for t in tasks if t[5] >= 0}
        assert not reads & set(writes)


def test_schedule_arguments_are_checked(ras):
    import ctypes as C
    L = ras.lib()
    fl, sl, ns = C.c_int(-1), C.c_int(-1), C.c_int(-1)
    assert L.ras_coarse_cr_schedule(0, None, 0, None, 0, C.byref(fl), C.byref(sl), C.byref(ns)) == ras.RAS_EINVAL
    # too small: lengths still reported
    assert L.ras_coarse_cr_schedule(9, None, 0, None, 0, C.byref(fl), C.byref(sl), C.byref(ns)) == ras.RAS_EINVAL
    fac, sol, nslot = ras.coarse_cr_schedule(9)
    assert (fl.value, sl.value, ns.value) == (len(fac), len(sol), nslot)
