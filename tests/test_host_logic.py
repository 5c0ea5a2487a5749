"""Host-side logic without a GPU: mesh validation and layout in libsesw, and the
multi-rank aggregation of the benchmark (two gloo ranks on the CPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2311_08241_gb300 import inputs as I
from paper_2311_08241_gb300 import sesw as S


def _check(mesh, pv=512):
    return S.sesw_mesh_check(mesh, pv)


@pytest.mark.parametrize("maker", [lambda: I.basin_case().mesh, lambda: I.channel_case().mesh,
                                   lambda: I.sphere_mesh(5), lambda: I.tiny_jittered_case().mesh])
def test_layout_of_valid_meshes(maker):
    m = maker()
    info = _check(m, 256)
    assert info["nv"] == m.nv and info["ne"] == m.ne
    assert info["npatch"] == -(-m.nv // 256)
    assert info["ne"] <= info["nslot"] <= 3 * info["ne"]
    assert info["max_patch_slots"] >= info["nslot"] / info["npatch"]


def test_hilbert_order_keeps_patches_compact():
    """Guest copies (elements on patch borders) are few with the space-filling-curve order and
    many when patches are cut from the lattice's row-major order."""
    m = I.channel_case().mesh
    hil = _check(m, 512)
    info_rm = S.sesw_mesh_check(_NoPos(m), 512)
    g_hil = (hil["nslot"] - hil["ne"]) / hil["ne"]
    g_rm = (info_rm["nslot"] - info_rm["ne"]) / info_rm["ne"]
    assert g_hil < 0.4 and g_rm > 2 * g_hil
    big = _check(m, 8192)
    assert (big["nslot"] - big["ne"]) / big["ne"] < 0.5 * g_hil


class _NoPos:
    def __init__(self, m):
        self.tri, self.xy, self.depth, self.coriolis = m.tri, m.xy, m.depth, m.coriolis
        self.pos = None
        self.nv, self.ne = m.nv, m.ne


def _bad(mutate):
    c = I.tiny_jittered_case()
    m = c.mesh
    b = I.Mesh(m.name, m.tri.copy(), m.xy.copy(), m.pos.copy(), m.depth.copy(), m.coriolis.copy())
    mutate(b)
    return b


@pytest.mark.parametrize("mutate,needle", [
    (lambda b: b.tri.__setitem__((2, 0), -1), "out of range"),
    (lambda b: b.tri.__setitem__((2, 1), b.tri[2, 0]), "repeats a vertex"),
    (lambda b: b.xy.__setitem__((0, 0, 0), np.nan), "non-finite coordinate"),
    (lambda b: b.depth.__setitem__(3, 0.0), "depth"),
    (lambda b: b.coriolis.__setitem__(1, np.inf), "Coriolis"),
])
def test_malformed_meshes_are_rejected(mutate, needle):
    with pytest.raises(S.SeswError) as ei:
        _check(_bad(mutate))
    assert ei.value.code == S.SESW_EINVAL and needle in str(ei.value)


def test_clockwise_triangle_rejected():
    c = I.tiny_jittered_case()
    m = c.mesh
    xy = m.xy.copy()
    xy[5, [1, 2]] = xy[5, [2, 1]]
    tri = m.tri.copy()
    b = I.Mesh(m.name, tri, xy, m.pos, m.depth, m.coriolis)
    with pytest.raises(S.SeswError, match="counter-clockwise"):
        _check(b)


def test_topology_errors_rejected():
    xy1 = np.array([[[0, 0], [1, 0], [0, 1]], [[1, 0], [0, 0], [0, -1]], [[0, 0], [1, 0], [1, 1]]], float) * 1e3
    tri = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    m = I.Mesh("t", tri, xy1, np.zeros((5, 3)), np.ones(5), np.zeros(3))
    with pytest.raises(S.SeswError, match="more than two"):
        _check(m)
    # two triangles walking a shared edge the same way
    tri2 = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    xy2 = np.array([[[0, 0], [1, 0], [0, 1]], [[0, 0], [1, 0], [0.5, 2]]], float) * 1e3
    m2 = I.Mesh("t", tri2, xy2, np.zeros((4, 3)), np.ones(4), np.zeros(2))
    with pytest.raises(S.SeswError, match="same direction"):
        _check(m2)
    # a vertex that no triangle uses
    m3 = I.Mesh("t", tri2[:1], xy2[:1], np.zeros((4, 3)), np.ones(4), np.zeros(1))
    with pytest.raises(S.SeswError, match="not a corner"):
        _check(m3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    slowest = bench.reduce_max(10.0 + rank, world, "cpu")
    bench.barrier(world)
    out.put((rank, slowest, bench.whole_job_value(1000, 40, 5, world, slowest)))
    dist.destroy_process_group()


def test_bench_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert res[0][2] == pytest.approx(2 * 1000 * 40 * 5 / 11e-3)


@pytest.mark.parametrize("maker", [lambda: I.channel_case(), lambda: I.basin_case(),
                                   lambda: I.ensemble_cases(nbasins=1, scale=0.05)[0]])
def test_courant_bound_is_an_upper_bound(maker):
    """The library's Courant bound is >= the true spectral radius of -div(g H0 grad) (scipy eigsh
    on the symmetrised lumped operator), and not far above it."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    case = maker()
    m = case.mesh
    info = _check(m, 512)
    xy, tri = m.xy, m.tri
    A = 0.5 * ((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
               - (xy[:, 2, 0] - xy[:, 0, 0]) * (xy[:, 1, 1] - xy[:, 0, 1]))
    G = np.zeros((m.ne, 3, 2))
    for k in range(3):
        d = xy[:, (k + 2) % 3] - xy[:, (k + 1) % 3]
        G[:, k, 0] = -d[:, 1] / (2 * A)
        G[:, k, 1] = d[:, 0] / (2 * A)
    w = A * m.depth[tri].mean(axis=1)
    r, c, v = [], [], []
    for a in range(3):
        for b in range(3):
            r.append(tri[:, a])
            c.append(tri[:, b])
            v.append(w * (G[:, a] * G[:, b]).sum(axis=1))
    K = sp.coo_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=(m.nv, m.nv)).tocsr()
    Av = np.zeros(m.nv)
    for k in range(3):
        np.add.at(Av, tri[:, k], A / 3)
    Dm = sp.diags(1 / np.sqrt(Av))
    lam = sla.eigsh(Dm @ K @ Dm, k=1, which="LA", return_eigenvectors=False)[0]
    assert lam <= info["stiffness_bound"] * (1 + 1e-9)
    assert info["stiffness_bound"] <= 2.0 * lam


# ---------------------------------------------------------------- optional caller tables

def _tables(mesh):
    """Edges and areas from the oracle's own mesh preparation (an independent derivation)."""
    from oracle import runner as orc

    om = orc.OracleMesh(mesh)
    ev, ee = om.edges()
    av, ae = om.areas()
    return (ev, ee), (av, ae)


def test_caller_edges_and_areas_are_accepted():
    m = I.tiny_jittered_case(nx=9, ny=7, seed=4).mesh
    edges, areas = _tables(m)
    base = S.sesw_mesh_check(m, 64)
    info = S.sesw_mesh_check(m, 64, edges=edges, areas=areas)
    assert info == base
    # any order of an edge's vertices and of its two triangles
    ev, ee = (x.copy() for x in edges)
    perm = np.random.default_rng(0).permutation(len(ev))
    S.sesw_mesh_check(m, 64, edges=(ev[perm][:, ::-1], ee[perm][:, ::-1]), areas=areas)


@pytest.mark.parametrize("what,needle", [
    ("area_e", "area_e"), ("area_v", "area_v"), ("edge_side", "triangles on its two sides"),
    ("edge_missing", "lists"), ("edge_twice", "listed twice"), ("edge_bogus", "not a side"),
    ("edge_half", "given together")])
def test_caller_tables_that_disagree_are_refused(what, needle):
    m = I.tiny_jittered_case(nx=9, ny=7, seed=4).mesh
    (ev, ee), (av, ae) = _tables(m)
    ev, ee, av, ae = ev.copy(), ee.copy(), av.copy(), ae.copy()
    edges, areas = (ev, ee), (av, ae)
    if what == "area_e":
        ae[5] *= 1.0 + 1e-9
    elif what == "area_v":
        av[3] *= 1.0 - 1e-9
    elif what == "edge_side":
        k = int(np.argmax(ee[:, 1] >= 0))
        ee[k, 1] = (ee[k, 1] + 1) % m.ne
    elif what == "edge_missing":
        edges = (ev[1:], ee[1:])
    elif what == "edge_twice":
        ev[1], ee[1] = ev[0], ee[0]
    elif what == "edge_bogus":
        a, b = ev[0]
        ev[0] = (a, next(v for v in range(m.nv) if v != a and not np.any(np.all(np.sort(ev, 1) == sorted((a, v)), 1))))
    elif what == "edge_half":
        edges = (ev, None)
    with pytest.raises(S.SeswError, match=needle) as e:
        S.sesw_mesh_check(m, 64, edges=edges, areas=areas)
    assert e.value.code == S.SESW_EINVAL


def test_bench_variants_run_on_the_channel():
    """The scheme and optional-term variants default to the channel workload; the batched
    ensemble and the surrogate refuse them."""
    import bench

    assert bench.parse([]).workload == "ensemble"
    assert bench.parse(["--scheme", "sesm"]).workload == "channel"
    assert bench.parse(["--visc", "auto"]).workload == "channel"
    assert bench.parse(["--freshwater", "2e-6", "--workload", "sphere"]).workload == "sphere"
    with pytest.raises(SystemExit):
        bench.parse(["--scheme", "sesm", "--workload", "ensemble"])


def test_bench_issue_roofline_and_profile_figures(tmp_path, monkeypatch):
    """The issue-bound roofline divides warp instructions by time against SMs x 4 x clock, and
    the committed kernel summaries are read only when their source hash matches, per layout."""
    import bench

    r = bench.roofline_issue("k", 2e-3, 1.2e9, 4e8, 3e10, 152, 2070.0, per="step")
    peak = 152 * 4 * 2070e6
    assert r["bound"] == "issue" and abs(r["peak"] - peak) < 1.0
    assert abs(r["achieved"] - 6e11) < 1.0 and abs(r["frac"] - 6e11 / peak) < 1e-12
    assert abs(r["dram"]["achieved_gbs"] - 200.0) < 1e-9
    assert abs(r["algorithmic"]["gbs"] - 15000.0) < 1e-6
    assert bench.roofline_issue("k", 1e-3, None, None, 1e9, 152, 2070.0)["frac"] is None

    h = bench.kernel_source_hash(("k_persistent",))
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(f"kernel_source_sha256_16: {h}\n\nlayout: a\nwarp_instructions_per_step: 5\n"
                               "dram_bytes_per_step: 7\n\nlayout: b\nwarp_instructions_per_step: 11\n")
    (prof / "stale.md").write_text("kernel_source_sha256_16: 0000000000000000\nwarp_instructions_per_launch: 3\n")
    real_join = bench.os.path.join
    monkeypatch.setattr(bench.os.path, "join",
                        lambda *a: str(prof / a[-1]) if len(a) == 3 and a[1] == "profiles" else real_join(*a))
    assert bench.profile_figures("x", ("k_persistent",), layout="a")["warp_instructions_per_step"] == 5.0
    assert bench.profile_figures("x", ("k_persistent",), layout="b")["warp_instructions_per_step"] == 11.0
    assert bench.profile_figures("x", ("k_persistent",), layout="c") is None
    assert bench.profile_figures("stale", ("k_persistent",)) is None


def test_bench_reference_arm_on_a_small_ensemble():
    """`bench.py --impl reference` times the oracle on the host cores and prints one JSON line with
    the reference keys (a tiny ensemble of the default recipe, one step)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--ensemble-basins",
                          "3", "--ensemble-scale", "0.03", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == line["metric"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
