"""A device-side wait that runs out: with the SIMT spin-wait limit set to 0 polls, the grid
barrier of the cooperative panel factorisation (and the bulge chase's progress flags)
expire at their first wait, the kernels record ELSI_ERR_TIMEOUT in the status word and
return, and the solve reports ELSI_ERR_TIMEOUT. The wait ends by its own limit: nothing is
faulted, trapped or hung, and the same handle then solves correctly with the default
limit restored (checked against the FP64 CPU oracle)."""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402

DEFAULT_LIMIT = 1 << 26


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_spin_wait_expires_then_handle_recovers():
    lib = egb.load()
    # n = 600 with b = 64: the first panels have more than 256 rows, so the panel
    # factorisation runs on several CTAs and its grid barrier has to wait
    p = ksinputs.cluster_problem(600, seed=51)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    H, S = dev(p.h), dev(p.s)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        assert lib.elsi_gb_set_spin_limit(0) == 0
        try:
            with pytest.raises(egb.ElsiError) as e:
                hd.dm_real(H.clone(), S)
        finally:
            assert lib.elsi_gb_set_spin_limit(DEFAULT_LIMIT) == 0
        assert e.value.code == 6  # ELSI_ERR_TIMEOUT
        assert "wait" in str(e.value)
        torch.cuda.synchronize()  # the context is still usable
        P, energy = hd.dm_real(H.clone(), S)
        W = hd.get_edm()
    assert rel(P.cpu().numpy(), ref["P"]) <= 1e-9
    assert rel(W.cpu().numpy(), ref["W"]) <= 1e-9
    assert abs(energy - ref["energy"]) <= 1e-9 * abs(ref["energy"])
