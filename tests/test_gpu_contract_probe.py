"""The tensor-core measurement of the interpolation stage (mf_contract_probe):
nodal values of 4 fields of 32 cells -> values and first reference
derivatives at the 27 Gauss points of Q2 (Section 3.1 sum factorisation),
by FP32 FMA sum factorisation, tcgen05 TF32 and tcgen05 3xTF32, against the
same contraction in FP64 with the oracle's tensor basis (oracle/basis.py).

Tolerances (max |error| / max |reference|): FP32 FMA and 3xTF32 carry FP32
rounding of a 27-term sum (<= 27 x 6e-8 relative per output), 1e-5 is the
FP32 apply bar; plain TF32 keeps 10 mantissa bits of each operand (2^-11
relative each), so 1e-2 bounds it and 1e-5 must not (the reason for variant 2)."""
import numpy as np
import pytest

from oracle.basis import tensor_basis, tensor_gauss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(u):
    pts, _ = tensor_gauss(2, 3)
    phi, dphi, _ = tensor_basis(2, 3, pts)             # [27 q, 27 a], [27 q, 27 a, 3]
    mats = [phi] + [dphi[:, :, d] for d in range(3)]
    M = np.concatenate(mats, axis=0)                     # [108, 27]
    return np.einsum("na,bafc->bnfc", M, u.astype(np.float64))


@pytest.mark.parametrize("blocks", [1, 148, 300])
def test_contract_probe_matches_fp64(blocks):
    from paper_2608_27423_b300 import contract_probe
    rng = np.random.default_rng(blocks)
    u = rng.uniform(-1, 1, (blocks, 27, 4, 32)).astype(np.float32)
    ref = _reference(u)
    ud = torch.tensor(u, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = {}
    for v in (0, 1, 2):
        out = torch.full((blocks, 108, 4, 32), float("nan"), dtype=torch.float32, device="cuda")
        contract_probe(v, ud, out, reps=1, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0, v
        got[v] = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got[v]).all(), v
    scale = np.abs(ref).max()
    e = {v: np.abs(got[v] - ref).max() / scale for v in got}
    print("max rel error fma %.2e tf32 %.2e 3xtf32 %.2e" % (e[0], e[1], e[2]))
    assert e[0] <= 1e-5 and e[2] <= 1e-5
    assert e[1] <= 1e-2


def test_contract_probe_repetitions_sum():
    """reps > 1: per (block, field, cell) the sum of all 108 outputs over the
    repetitions, i.e. reps x the row sum of the single contraction."""
    from paper_2608_27423_b300 import contract_probe
    rng = np.random.default_rng(5)
    blocks, reps = 148, 6
    u = rng.uniform(-1, 1, (blocks, 27, 4, 32)).astype(np.float32)
    ref = reps * _reference(u).sum(axis=1)              # [blocks, 4, 32]
    ud = torch.tensor(u, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for v in (0, 2):
        out = torch.zeros((blocks, 4, 32), dtype=torch.float32, device="cuda")
        contract_probe(v, ud, out, reps=reps, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        got = out.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), v
