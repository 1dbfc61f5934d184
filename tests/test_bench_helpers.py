"""bench.py's host-side helpers: the gate that reports a committed ncu
capture's DRAM traffic only while the kernel's sources are unchanged, the
algorithmic-bytes model, and the count of our kernel launches per step."""
import hashlib
import os
import types

import bench


def _write_profile(root, name, sources, nbytes, shape=None, tamper=False):
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(root, "paper_1411_2141_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    if tamper:
        digest = ("0" if digest[0] != "0" else "1") + digest[1:]
    lines = [f"- source sha256 ({', '.join(sources)}): {digest}",
             f"- DRAM bytes per launch: {nbytes}"]
    if shape:
        lines.append(f"- team shape (ctas,block,blocks_per_sm): {shape[0]},{shape[1]},{shape[2]}")
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", name), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def _fake_root(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1411_2141_gb300", "csrc")
    dst = tmp_path / "paper_1411_2141_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("device_common.cuh", "iterate.cu"):
        with open(os.path.join(src, f), "rb") as a, open(dst / f, "wb") as b:
            b.write(a.read())
    return str(tmp_path)


def test_traffic_is_reported_only_for_the_profiled_sources(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    srcs = ["device_common.cuh", "iterate.cu"]
    _write_profile(root, "a.md", srcs, 12345)
    assert bench.profiled_traffic(("a.md", srcs)) == 12345
    _write_profile(root, "b.md", srcs, 12345, tamper=True)
    assert bench.profiled_traffic(("b.md", srcs)) is None          # sources changed since
    assert bench.profiled_traffic(("missing.md", srcs)) is None
    _write_profile(root, "c.md", srcs, 777, shape=(8, 256, 2))
    assert bench.profiled_traffic(("c.md", srcs), (8, 256, 2)) == 777
    assert bench.profiled_traffic(("c.md", srcs), (4, 512, 1)) is None   # another team shape
    with open(os.path.join(root, "paper_1411_2141_gb300", "csrc", "iterate.cu"), "a") as fh:
        fh.write("// edit\n")
    assert bench.profiled_traffic(("a.md", srcs)) is None          # a kernel source was edited


def test_algorithmic_bytes_model():
    n_v, n_t, nnz = 20000, 39870, 2 * 59869
    s0 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S0", 0.0)
    s1_0 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S1", 0.0)
    s1_4 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S1", 4.0)
    s2_4 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S2", 4.0)
    # linear in the CG count, S2 reads the stored matrix values on top of S1
    s1_8 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S1", 8.0)
    assert abs((s1_8 - s1_4) - (s1_4 - s1_0)) < 1e-6 * s1_8
    assert s2_4 > s1_4 > s1_0 > 0 and s0 > 0
    # per node: sample 24 B, force ~60 B, S0 update ~52 B, a CG step ~140-200 B
    assert 100 <= s0 / n_v <= 200
    assert 140 <= (s1_4 - s1_0) / 4 / n_v <= 220
    # proportional to the mesh size
    s1_big = bench.algorithmic_bytes_per_iteration(2 * n_v, 2 * n_t, 2 * nnz, "S1", 4.0)
    assert abs(s1_big - 2 * s1_4) < 1e-6 * s1_big
    # Chebyshev: the first step is in the force phase; each further step moves
    # the graph, x, b, d and the Jacobi entries (~80 B/node), far less than a
    # CG step (the CG state of every neighbour)
    c1 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S1", 1.0, "chebyshev")
    c5 = bench.algorithmic_bytes_per_iteration(n_v, n_t, nnz, "S1", 5.0, "chebyshev")
    assert 60 <= (c5 - c1) / 4 / n_v <= 100
    assert c1 > s1_0 - 1e-6 and c5 < s1_4


def test_solver_names():
    ns = types.SimpleNamespace
    assert bench.solver_of(ns(mode="S1", solver="auto")) == "chebyshev"
    assert bench.solver_of(ns(mode="S1", solver="cg")) == "cg"
    assert bench.solver_of(ns(mode="S2", solver="auto")) == "cg"
    assert bench.solver_of(ns(mode="S0", solver="auto")) == "none"


def test_launch_counts_match_the_measured_launch_lists():
    # one 512^2 registration in the ncu launch list: 4 prefilter passes, the
    # node samples, pixel fill + map, the iteration kernel + its energy sums,
    # the warp's affine records, the warp and the MSD sum
    args = types.SimpleNamespace(coeff="fp32")
    assert bench.launches_per_registration(args, 200) == 12
    assert bench.launches_per_registration(args, 1100) == 14            # two 1024-iteration launches
    assert bench.launches_per_registration(types.SimpleNamespace(coeff="bf16"), 200) == 13
    assert bench.ADJOINT_LAUNCHES == 7
    assert bench.adjoint_launches(20, 0) == 7 and bench.adjoint_launches(20, 20) == 7
    assert bench.adjoint_launches(20, 5) == 4 + 5 * 4     # 4 segments


def test_operator_bytes():
    # S1: columns, x and y; S2 adds the stored values and diagonal
    assert bench.operator_bytes(10, 60, "S1") == 4 * 60 + 16 * 10
    assert bench.operator_bytes(10, 60, "S2") == bench.operator_bytes(10, 60, "S1") + 4 * 60 + 40
