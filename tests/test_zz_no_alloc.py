"""The allocation-free energy entry point (collected last on purpose).

ddlpb_energy_noalloc serves callers that cannot allocate device memory when they
need the energy; it reads the caller's charges and solution vector and keeps its
partial sums in a fixed device array of the library.  Its result must equal the
context-based ddlpb_energy, call after call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_00552_gb300 as G
from paper_2203_00552_gb300 import _binding, synth

pytestmark = pytest.mark.gpu

KAPPA = synth.KAPPA_PER_ANGSTROM / synth.ANGSTROM_TO_BOHR


def _solved(n, seed, lmax, nleb):
    c, r, q = synth.molecule(n, seed, "chain")
    ctx = G.Context(c, r, q, synth.EPS_SOLVENT, KAPPA, lmax, nleb, tol=1e-12)
    ctx.solve()
    X = torch.empty(ctx.nvec, dtype=torch.float64, device="cuda:0")
    ctx.vector(1, X)
    return ctx, torch.tensor(q, device="cuda:0"), X


def test_energy_noalloc_matches_context_energy_twice():
    big, qb, Xb = _solved(40, 6, 4, 50)
    small, qs, Xs = _solved(9, 2, 3, 26)
    Eb, Es = big.energy(), small.energy()
    # two calls in a row on each input, alternating sizes so that stale scratch would show
    for _ in range(2):
        e1 = _binding.energy_noalloc(40, 4, qb, Xb)
        e2 = _binding.energy_noalloc(9, 3, qs, Xs)
        assert abs(e1 - Eb) <= 1e-12 * abs(Eb)
        assert abs(e2 - Es) <= 1e-12 * abs(Es)
    # device output on a side stream
    s = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    lib = _binding.library()
    st = lib.ddlpb_energy_noalloc(40, 4, _binding._ptr(qb), _binding._ptr(Xb), _binding._ptr(out),
                                  _binding.C.c_void_p(s.cuda_stream))
    assert st == 0
    assert abs(float(out) - Eb) <= 1e-12 * abs(Eb)


def test_energy_noalloc_rejects_sizes_beyond_its_scratch():
    q = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    X = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(G.DDLPBError) as e:
        _binding.energy_noalloc(1048577, 0, q, X)
    assert e.value.status == 1
    with pytest.raises(G.DDLPBError) as e:
        _binding.energy_noalloc(0, 0, q, X)
    assert e.value.status == 1
