"""Per-call metrics log (mf_log_open): host-side calls (mesh generation,
checkpoints) append one parseable JSON object per line with their status and
sizes; turning the log off stops the records."""
import json

import numpy as np


def test_log_records_host_calls(tmp_path):
    from paper_2608_27423_b300 import log_open, rotor_stator_mesh, save_checkpoint, load_checkpoint, MfError
    path = tmp_path / "calls.jsonl"
    log_open(path)
    try:
        mesh = rotor_stator_mesh(d=2, k=2, m=4, n_r=2, n_s=3)
        u = np.zeros((mesh.n_nodes, 3))
        save_checkpoint(tmp_path / "c.ckpt", mesh, u, step=3, t=0.03, theta=0.5, dt=0.01, nu=0.1, omega=1.0)
        load_checkpoint(tmp_path / "c.ckpt", mesh)
        try:
            load_checkpoint(tmp_path / "missing.ckpt", mesh)
        except MfError:
            pass
    finally:
        log_open(None)
    rotor_stator_mesh(d=2, k=1, m=2, n_r=1, n_s=1)          # not logged any more
    recs = [json.loads(line) for line in open(path)]
    calls = [r["call"] for r in recs]
    assert calls[0] == "mf_mesh_rotor_stator" and calls.count("mf_mesh_rotor_stator") == 1
    assert calls[1:] == ["mf_checkpoint_write", "mf_checkpoint_read", "mf_checkpoint_read"]
    g = recs[0]
    assert (g["d"], g["k"], g["n_nodes"], g["n_cells"], g["n_R"]) == (2, 2, mesh.n_nodes, mesh.n_cells, 16)
    assert recs[1]["status"] == 0 and recs[1]["step"] == 3 and recs[2]["theta"] == 0.5
    assert recs[3]["status"] == 1 and "step" not in recs[3]
    assert all(r["seconds"] >= 0 for r in recs)
