"""CPU check of the tracer's BVH build (host code shared with the library): the harness
tests/bvh_check.cpp compiles the library's builder and checks the invariants the GPU
traversal relies on, on the synthetic cities and on degenerate triangle sets."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2501_13382_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("bvh") / "bvh_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2501_13382_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                    os.path.join(HERE, "bvh_check.cpp"), "-o", exe], check=True)
    return exe


def _run(harness, tmp_path, tris):
    tris = np.ascontiguousarray(np.asarray(tris, np.float64).reshape(-1, 9))
    path = str(tmp_path / "tris.bin")
    with open(path, "wb") as f:
        f.write(np.int64(tris.shape[0]).tobytes())
        f.write(tris.tobytes())
    r = subprocess.run([harness, path], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
    return r.stdout


def _degenerate(name):
    rng = np.random.default_rng(5)
    if name == "identical":                     # every centroid equal: median splits only
        return np.tile([0.0, 0, 0, 1, 0, 0, 0, 1, 0], (300, 1))
    if name == "collinear":                     # centroids on one line
        x = np.arange(257, dtype=float)
        t = np.zeros((257, 9))
        t[:, 0], t[:, 3], t[:, 6] = x, x + 0.5, x
        t[:, 4], t[:, 7] = 0.0, 0.0
        t[:, 8] = 1.0
        return t
    if name == "soup":                          # random triangles, widely varying sizes
        c = rng.uniform(-500, 500, (5000, 1, 3))
        return (c + rng.normal(size=(5000, 3, 3)) * rng.uniform(0.01, 30, (5000, 1, 1))).reshape(-1, 9)
    if name == "clustered":                     # two far clusters, one much denser
        a = rng.normal(size=(3000, 9)) * 0.5
        b = rng.normal(size=(40, 9)) * 0.5 + 1e4
        return np.concatenate([a, b])
    raise KeyError(name)


@pytest.mark.parametrize("n", [1, 2, 4, 5, 9, 17])
def test_bvh_small_scenes(harness, tmp_path, n):
    tris, _ = I.box_triangles(8.0, 20.0, -6.0, 6.0, 15.0)
    tris = np.concatenate([tris, tris + 30.0])[:n]
    _run(harness, tmp_path, tris)


@pytest.mark.parametrize("which", ["city", "big_city"])
def test_bvh_synthetic_cities(harness, tmp_path, which):
    sc = I.city_scene(I.SEED_BASE + 3)[0] if which == "city" else \
        I.city_scene(I.SEED_BASE + 6, n_side=32, extent=2000.0)[0]
    out = _run(harness, tmp_path, sc.tri_xyz)
    depth = int(out.split("depth=")[1])
    assert depth <= 2 * int(np.ceil(np.log2(sc.n_tri)))      # SAH keeps it shallow here


@pytest.mark.parametrize("name", ["identical", "collinear", "soup", "clustered"])
def test_bvh_degenerate_sets(harness, tmp_path, name):
    _run(harness, tmp_path, _degenerate(name))


@pytest.mark.parametrize("old,new", [
    ("bounds(lo, mid, nd.box[0]);", "bounds(lo, mid - 1, nd.box[0]);"),        # box misses a triangle
    ("return -(int32_t)(first * 8 + (count - 1)) - 1;", "return -(int32_t)(first * 8 + count) - 1;"),
    ("if (hi - lo <= kBvhLeaf) return leaf_ref(lo, hi - lo);",
     "if (hi - lo <= kBvhLeaf + 2) return leaf_ref(lo, hi - lo);"),           # oversized leaves
])
def test_planted_builder_mistakes_are_caught(tmp_path, old, new):
    """The checker is not vacuous: copies of the builder with a plausible slip fail it."""
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = open(os.path.join(ROOT, "paper_2501_13382_gb300", "csrc", "bvh_build.h")).read()
    assert src.count(old) == 1, old
    inc = tmp_path / "inc"
    inc.mkdir()
    (inc / "bvh_build.h").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "paper_2501_13382_gb300", "csrc", "gbt_internal.h"), inc)
    exe = str(tmp_path / "bvh_check_mut")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", str(inc), "-I", os.path.join(ROOT, "include"),
                    "-I", CUDA_INC, os.path.join(HERE, "bvh_check.cpp"), "-o", exe], check=True)
    # random triangles: every box differs (the city's faces are pairs of triangles with the
    # same box, which would hide a box that misses one of them)
    tris = np.ascontiguousarray(_degenerate("soup"), np.float64)
    path = str(tmp_path / "tris.bin")
    with open(path, "wb") as f:
        f.write(np.int64(tris.shape[0]).tobytes())
        f.write(tris.tobytes())
    r = subprocess.run([exe, path], capture_output=True, text=True)
    assert r.returncode != 0 and "FAIL" in r.stdout, r.stdout
