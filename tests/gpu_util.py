"""Helpers shared by the GPU parity tests."""
import numpy as np
import pytest

try:
    import torch
except Exception:  # pragma: no cover
    torch = None


def need_gpu():
    if torch is None or not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def assert_within(y, ref, bound, rel, what=""):
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert y.shape == ref.shape, (what, y.shape, ref.shape)
    err = np.abs(y - ref)
    lim = rel * np.asarray(bound, dtype=np.float64)
    bad = np.nonzero(~(err <= lim))[0]
    assert bad.size == 0, (f"{what}: {bad.size} entries outside {rel}*sum|a x|; first at {bad[:5]}: "
                           f"got {y[bad[:5]]}, want {ref[bad[:5]]}, bound {lim[bad[:5]]}")


def assert_bitexact(y, ref, what=""):
    y = np.asarray(y)
    ref = np.asarray(ref)
    assert y.shape == ref.shape, (what, y.shape, ref.shape)
    bad = np.nonzero(y != ref)[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches; first at {bad[:5]}: {y[bad[:5]]} vs {ref[bad[:5]]}"
