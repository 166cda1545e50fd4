"""The C ABI from plain C: include/mf.h compiles as C99 with warnings as
errors, and a C program linked against libmf.so drives the host-side entry
points (mesh generator, mesh read-back, checkpoint round trip, argument
checks); its mesh sizes equal the Python binding's."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_uses_the_library(tmp_path):
    from paper_2608_27423_b300 import build, rotor_stator_mesh
    so = build.build()
    exe = tmp_path / "demo"
    libdir = os.path.dirname(so)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "host_abi_demo.c"), "-o", str(exe), os.path.join(libdir, "libmf.so"),
           f"-Wl,-rpath,{libdir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe), str(tmp_path / "c.ckpt")], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = dict(line.split(" ", 1) for line in out.stdout.strip().splitlines())
    mesh = rotor_stator_mesh(d=3, k=2, m=4, n_r=2, n_s=2, n_z=2, blades=2)
    d, k, nn, nc, n_R, n_z = map(int, lines["sizes"].split())
    assert (d, k, nn, nc, n_R, n_z) == (3, 2, mesh.n_nodes, mesh.n_cells, mesh.n_R, mesh.n_z)
    moving = int(lines["moving_wall_nodes"].split()[0])
    assert moving == int((mesh.wall == 2).sum()) and moving > 0
    assert lines["checkpoint"] == "ok" and lines["args"] == "ok"
