"""Host-only checks of the binding's *_dev wrappers: tensors of the wrong dtype,
length or layout, or not on the current CUDA device, are rejected with
ValueError before anything reaches the library (a wrong tensor passed on as a
raw pointer would make a kernel read or write out of bounds)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _bare_solver(n):
    # a Solver object without a handle: the checks run before any library call
    import paper_1611_06721_gb300.binding as b
    s = object.__new__(b.Solver)
    s.h, s.lib = None, None
    s.n = n
    s.n_layout = 3 * n ** 3
    s.n_c = 5
    return s


def test_noalloc_wrapper_rejects_wrong_tensors():
    from paper_1611_06721_gb300.binding import pcg_solve_noalloc
    n = 4
    mask = torch.zeros(n ** 3, dtype=torch.uint8)
    b = torch.zeros(3 * n ** 3, dtype=torch.float64)
    x = torch.zeros(3 * n ** 3, dtype=torch.float64)
    cases = [
        (mask, b.float(), x, "float64"),                              # FP32 right-hand side
        (mask, b[: n ** 3], x, "values"),                             # n^3 instead of 3 n^3
        (mask.to(torch.int32), b, x, "uint8"),                        # wrong mask type
        (mask, b, torch.zeros(2 * 3 * n ** 3, dtype=torch.float64)[::2], "contiguous"),
        (mask, b, x, "CUDA"),                                         # host tensors
        (mask, b, np.zeros(3 * n ** 3), "torch tensor"),
    ]
    for m, bb, xx, what in cases:
        with pytest.raises(ValueError, match=what):
            pcg_solve_noalloc(n, 1e-3, 1.0, m, bb, xx)


def test_handle_dev_wrappers_reject_wrong_tensors():
    s = _bare_solver(4)
    L = s.n_layout
    good = torch.zeros(L, dtype=torch.float64)
    with pytest.raises(ValueError, match="float64"):
        s.pcg_solve_dev(good.float(), good)
    with pytest.raises(ValueError, match="values"):
        s.pcg_solve_dev(good[: L // 3], good)
    with pytest.raises(ValueError, match="CUDA"):
        s.pcg_solve_dev(good, good.clone())
    with pytest.raises(ValueError, match="values"):
        s.apply_kn_dev(good, torch.zeros(L - 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="values"):
        s.set_state_dev(torch.zeros(s.n_c + 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        s.get_state_dev(torch.zeros(s.n_c, dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA"):
        s.get_state_dev(torch.zeros(s.n_c, dtype=torch.float64))


def test_get_state_rejects_a_wrong_output_buffer():
    # get_state(out=...) writes a_c into the caller's host array: only a writeable
    # C-contiguous float64 array of n_c values is accepted
    s = _bare_solver(4)
    bad = [np.zeros(s.n_c, dtype=np.float32), np.zeros(s.n_c + 1), np.zeros(2 * s.n_c)[::2], [0.0] * s.n_c]
    ro = np.zeros(s.n_c)
    ro.flags.writeable = False
    for out in bad + [ro]:
        with pytest.raises(ValueError, match="float64"):
            s.get_state(out=out)
