"""Rank-sweep labels of the learned proposer with one sketch per tensor: the
sketch and projection at the largest K of the sweep, every smaller K taken
as the leading block of that projection, and TR-ALS run on the small
projected tensors only (proposer.nested_rank_sweep), against the
sweep that decomposes the whole tensor again for every R
(proposer.rank_sweep_labels)."""
import numpy as np
import pytest
import torch

from paper_1901_01652_gb300 import proposer as pp
from paper_1901_01652_gb300 import rtr, workloads

pytestmark = pytest.mark.gpu

R_SWEEP = list(range(1, 8))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1901_01652_gb300 import build
    build.build()
    rtr.lib()


def _tensors(specs):
    Xs, Ss = [], []
    for dims, r, snr, seed in specs:
        R = [r] * len(dims)
        cores = [torch.from_numpy(c).cuda() for c in workloads.tr_cores(dims, R, seed)]
        S = torch.empty(dims, dtype=torch.float32, device="cuda")
        work = torch.empty(rtr.rtr_reconstruct_work_bytes(dims, R), dtype=torch.uint8, device="cuda")
        rtr.rtr_reconstruct(dims, R, cores, "fp32", S, work)
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        sigma = workloads.snr_sigma(float(torch.linalg.vector_norm(S, dtype=torch.float64)), S.numel(), snr)
        Xs.append(S + sigma * torch.randn(dims, generator=g, device="cuda"))
        Ss.append(S)
    return Xs, Ss


def test_nested_sweep_reproduces_the_full_sweep():
    specs = workloads.proposer_shapes(12, seed=2024)
    Xs, Ss = _tensors(specs)
    labels, table = pp.rank_sweep_labels(Xs, Ss, R_SWEEP, 1e-2, seed=5)
    # tensor t of rank_sweep_labels' batches runs with seed 5 + (its index in its order group)
    order_index, seen = [], {}
    for X in Xs:
        order_index.append(seen.get(X.dim(), 0))
        seen[X.dim()] = order_index[-1] + 1
    for t in range(len(Xs)):
        lab, errs = pp.nested_rank_sweep(Xs[t], Ss[t], R_SWEEP, 1e-2, seed=5 + order_index[t])
        assert lab == labels[t], (t, lab, labels[t])
        # the same TR-ALS from the same start on P_K blocks that agree to
        # rounding: equal errors up to the label; above it (R beyond the
        # tensor's rank) the fit is not unique and only its size is compared
        j = R_SWEEP.index(lab) + 1
        np.testing.assert_allclose(errs[:j], table[:j, t], rtol=1e-3, atol=1e-5, err_msg=str(t))
        assert np.all((errs[j:] <= 1e-2) == (table[j:, t] <= 1e-2)), t
