"""Checkpoint / resume files (mf_checkpoint_write / mf_checkpoint_read, host
code, no GPU): exact round trip of the BDF state and counters, a JSON header
that standard parsers read, and rejection of another mesh, a truncated file
and a damaged header."""
import json

import numpy as np
import pytest

import synth


def _state(mesh, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((mesh.n_nodes, mesh.d + 1))


@pytest.mark.parametrize("bdf", [1, 2])
def test_round_trip_is_exact(tmp_path, bdf):
    from paper_2608_27423_b300 import save_checkpoint, load_checkpoint
    mesh = synth.rotor_stator_mesh(3, 2, 4, 2, 2, 3, blades=2)
    un, unm1 = _state(mesh, 1), _state(mesh, 2)
    path = tmp_path / "run.ckpt"
    save_checkpoint(path, mesh, un, unm1 if bdf == 2 else None, step=17, t=0.034, theta=0.1234567890123,
                    dt=0.002, nu=1.0 / (4000 * np.pi), omega=1.0)
    assert not (tmp_path / "run.ckpt.tmp").exists()
    info, a, b = load_checkpoint(path, mesh)
    assert info["bdf"] == bdf and info["step"] == 17
    assert info["t"] == 0.034 and info["theta"] == 0.1234567890123 and info["dt"] == 0.002
    assert info["nu"] == 1.0 / (4000 * np.pi) and info["omega"] == 1.0
    assert np.array_equal(a, un)
    if bdf == 2:
        assert np.array_equal(b, unm1)
    else:
        assert b is None
    header = json.loads(open(path, "rb").readline())
    assert header["format"] == "mf-checkpoint-1" and header["n_nodes"] == mesh.n_nodes
    assert header["blobs"] == bdf and header["values_per_blob"] == mesh.n_dofs
    assert path.stat().st_size == len(open(path, "rb").readline()) + 8 * mesh.n_dofs * bdf


def test_rejects_other_mesh_and_damaged_files(tmp_path):
    from paper_2608_27423_b300 import save_checkpoint, load_checkpoint, MfError
    mesh = synth.rotor_stator_mesh(2, 2, 4, 2, 3)
    path = tmp_path / "a.ckpt"
    save_checkpoint(path, mesh, _state(mesh, 3), _state(mesh, 4), step=1, t=0.01, theta=0.0, dt=0.01, nu=0.01,
                    omega=1.0)
    # same sizes, other coordinates: the fingerprint differs
    other = synth.rotor_stator_mesh(2, 2, 4, 2, 3, R=0.45)
    assert other.n_nodes == mesh.n_nodes
    with pytest.raises(MfError):
        load_checkpoint(path, other)
    with pytest.raises(MfError):
        load_checkpoint(path, synth.rotor_stator_mesh(2, 2, 5, 2, 3))
    raw = open(path, "rb").read()
    (tmp_path / "short.ckpt").write_bytes(raw[:-8])
    with pytest.raises(MfError):
        load_checkpoint(tmp_path / "short.ckpt", mesh)
    (tmp_path / "bad.ckpt").write_bytes(raw.replace(b"mf-checkpoint-1", b"mf-checkpoint-9", 1))
    with pytest.raises(MfError):
        load_checkpoint(tmp_path / "bad.ckpt", mesh)
    with pytest.raises(MfError):
        load_checkpoint(tmp_path / "missing.ckpt", mesh)
    with pytest.raises(MfError):
        save_checkpoint(path, mesh, _state(mesh, 3)[:-1], step=1, t=0.0, theta=0.0, dt=0.01, nu=0.01, omega=1.0)
