"""The library's P2 reference tables (csrc/p2_tables.cpp, compiled here with the host compiler)
against the P2 oracle: the element mass and the facet mass and triple products that the P2
membrane kernels read from constant memory."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import p2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("p2t") / "p2_tables_dump")
    csrc = os.path.join(ROOT, "paper_2403_04491_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", csrc,
                    os.path.join(ROOT, "tests", "c", "p2_tables_dump.cpp"), os.path.join(csrc, "p2_tables.cpp"),
                    "-o", exe], check=True)
    out = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        name, d, *vals = line.split()
        out[(name, int(d))] = np.array([float(v) for v in vals])
    return out


@pytest.mark.parametrize("d", [2, 3])
def test_p2_reference_tables_match_oracle(tables, d):
    n = (d + 1) * (d + 2) // 2
    nf = d * (d + 1) // 2
    np.testing.assert_allclose(tables[("mass", d)].reshape(n, n), p2.local_mass(d), rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(tables[("fmass", d)].reshape(nf, nf), p2.local_mass(d - 1), rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(tables[("ftriple", d)].reshape(nf, nf, nf), p2.local_triple(d - 1), rtol=1e-14,
                               atol=1e-17)
    # the facet triple products are symmetric in their three indices (the kernels rely on it)
    W = tables[("ftriple", d)].reshape(nf, nf, nf)
    for perm in ((1, 0, 2), (0, 2, 1), (2, 1, 0)):
        assert np.array_equal(W, W.transpose(perm))
    # 2D: 3 vertex-vertex pairs x 4 terms + 9 vertex-edge x 4 + 3 edge-edge x 4; 3D likewise (180)
    assert int(tables[("nterms", d)][0]) == {2: 60, 3: 180}[d]
