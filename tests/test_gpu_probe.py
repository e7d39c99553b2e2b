"""The issue-rate probes behind the epilogue-pipe rooflines run and write bounded values:
the FMA chains a <- a m + c with 0 < m < 1 stay in (0, 2), the sine chains a <- 3 sin(a)
stay in [-3, 3]."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])
def test_probe_runs(kind):
    from paper_2604_25936_gb300 import binding as b
    nb = 4
    sink = torch.full((nb * b.PROBE_THREADS,), float("nan"), device="cuda")
    b.probe_rate(kind, nb, 1000, sink)
    torch.cuda.synchronize()
    v = sink.cpu()
    assert torch.isfinite(v).all()
    if kind == b.PROBE_FFMA:
        assert ((v > 0) & (v < 2 * b.PROBE_CHAINS)).all()
    else:
        assert (v.abs() <= 3 * b.PROBE_CHAINS).all()
