"""Host-side argument checks of the allocation-free Gram SpMV binding (gram_spmv_static): every
input that would make the raw-pointer entry point read or write past a buffer raises
ValueError before the library is called.  Runs without a GPU: the library is never reached."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def binding():
    from paper_2607_07485_b300 import build
    build.build()
    from paper_2607_07485_b300 import lsamg
    return lsamg


def _good(ne=3, m=2, nT=4, n=10):
    return (torch.zeros((ne, nT), dtype=torch.int32), torch.zeros((ne, m, nT), dtype=torch.float64),
            torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64))


def _raises(binding, args, match, monkeypatch):
    called = []
    monkeypatch.setattr(binding, "_check", lambda *a, **k: called.append(a))
    with pytest.raises(ValueError, match=match):
        binding.gram_spmv_static(*args)
    assert not called


@pytest.mark.parametrize("which,bad,match", [
    (0, lambda t: t.to(torch.int64), "elem_dofs must be torch.int32"),
    (1, lambda t: t.to(torch.float32), "G must be torch.float64"),
    (2, lambda t: t.to(torch.float32), "x must be torch.float64"),
    (3, lambda t: t.to(torch.float32), "y must be torch.float64"),
    (1, lambda t: t.transpose(1, 2), "G must be contiguous"),
    (2, lambda t: torch.zeros(20, dtype=torch.float64)[::2], "x must be contiguous"),
    (1, lambda t: t.reshape(t.shape[0], -1), r"G must be \[n_elems"),
    (1, lambda t: torch.zeros((2, 2, 4), dtype=torch.float64), r"G must be \[n_elems"),
    (1, lambda t: torch.zeros((3, 2, 5), dtype=torch.float64), r"G must be \[n_elems"),
    (3, lambda t: torch.zeros(9, dtype=torch.float64), "same length"),
    (0, lambda t: t.reshape(-1), "elem_dofs must be 2-D"),
])
def test_bad_input_raises_before_the_call(binding, monkeypatch, which, bad, match):
    args = list(_good())
    args[which] = bad(args[which])
    _raises(binding, args, match, monkeypatch)


def test_host_tensors_are_refused(binding, monkeypatch):
    # well-formed but on the host: the entry point takes device pointers only
    _raises(binding, list(_good()), "CUDA", monkeypatch)
