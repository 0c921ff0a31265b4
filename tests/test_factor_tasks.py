"""Host logic of the block Cholesky (Section 2: the damped normal equations are solved by a
Cholesky factorisation): the task orders the factor kernels claim, read back through the C-ABI
(ds_factor_tasks, no GPU). Every block is produced exactly once and every task comes after the
tasks whose results it reads, which is what keeps the persistent kernels free of deadlock."""
import pytest


@pytest.fixture(scope="module")
def d():
    from paper_2007_08576_gb300 import build, defsolve
    defsolve.lib(build.build())
    return defsolve


def needs(ty, i, j):
    """Results a task reads, from the left-looking recurrences L_jj L_jj^T = A_jj -
    sum_{k<j} L_jk L_jk^T and L_ij = (A_ij - sum_{k<j} L_ik L_jk^T) L_jj^-T."""
    if ty == 0:
        return {("L", j, k) for k in range(j)}
    if ty == 1:
        return ({("L", i, k) for k in range(j)} | {("L", j, k) for k in range(j)} |
                {("D", j)})
    j1 = j + 1
    rows = [i] if ty == 2 else [i, i + 1]
    need = ({("L", j, k) for k in range(j)} | {("L", j1, k) for k in range(j)} |
            {("D", j), ("D", j1), ("L", j1, j)})
    for r in rows:
        need |= {("L", r, k) for k in range(j)}
    return need


def gives(ty, i, j):
    if ty == 0:
        return [("D", j)]
    if ty == 1:
        return [("L", i, j)]
    if ty == 2:
        return [("L", i, j), ("L", i, j + 1)]
    return [("L", i, j), ("L", i, j + 1), ("L", i + 1, j), ("L", i + 1, j + 1)]


@pytest.mark.parametrize("paired", [0, 1, 2])
def test_orders_are_topological_and_complete(d, paired):
    for nb in range(1, 41):
        tasks = d.ds_factor_tasks(nb, paired)
        have, made = set(), []
        for ty, i, j in tasks.tolist():
            assert ty in ((0, 1), (0, 1, 2), (0, 1, 2, 3))[paired]
            missing = needs(ty, i, j) - have
            assert not missing, (nb, (ty, i, j), sorted(missing)[:3])
            for g in gives(ty, i, j):
                assert g not in have, (nb, g)          # produced once
                have.add(g)
            made.append((ty, i, j))
        want = {("D", j) for j in range(nb)} | {("L", i, j) for i in range(nb) for j in range(i)}
        assert have == want, nb


def test_single_order_looks_ahead_one_column(d):
    """DIAG(j + 1) is claimed right after OFF(j + 1, j), ahead of the rest of column j."""
    nb = 9
    tasks = [tuple(t) for t in d.ds_factor_tasks(nb).tolist()]
    for j in range(nb - 2):
        at = tasks.index((1, j + 1, j))
        assert tasks[at + 1] == (0, j + 1, j + 1)
        assert tasks.index((0, j + 1, j + 1)) < tasks.index((1, j + 2, j))


def test_bad_arguments(d):
    with pytest.raises(d.DsError):
        d.ds_factor_tasks(0)
    import ctypes
    n = ctypes.c_int32()
    assert d.lib().ds_factor_tasks(4, 3, None, 0, ctypes.byref(n)) == d.DS_ERR_ARG
    assert d.lib().ds_factor_tasks(4, 0, None, 5, ctypes.byref(n)) == d.DS_ERR_ARG
    assert d.lib().ds_factor_tasks(4, 0, None, 0, None) == d.DS_ERR_ARG
    assert d.lib().ds_factor_tasks(4, 0, None, 0, ctypes.byref(n)) == 0 and n.value == 10
