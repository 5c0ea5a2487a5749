"""Pick the execution layout of a mesh (or batch) by timing it on the GPU.

Candidates are the persistent kernel with 1, 2 or 4 resident blocks per SM, in
its automatic form and with every pack streamed, and the per-substep graph with
several patch sizes and block sizes. Each candidate is
uploaded through the C-ABI and timed with CUDA events on a few baroclinic steps
of the actual workload. A layout the mesh does not fit is skipped. The result
is the fastest candidate, plus the whole table so callers can report it.
"""
from __future__ import annotations

import dataclasses
import statistics

import numpy as np

from . import sesw as S

# three blocks per SM (320 threads at most) were measured slower on every workload here: the
# block size forces four slots per thread where two blocks of 512 take three
PERSISTENT_BLOCKS = (1, 2, 4)
GRAPH_PATCHES = (128, 256, 512, 1024)
GRAPH_THREADS = (128, 256, 512)
WAVE_BLOCKS_PER_SM = (2, 4, 8)


def wave_patch_sizes(nv_max, nsm, blocks_per_sm=WAVE_BLOCKS_PER_SM):
    """Graph-mode patch sizes that make the largest mesh exactly one wave of blocks when
    `k` blocks of the substep kernel are resident per SM (a partial second wave of a
    latency-bound kernel costs nearly a full one)."""
    return tuple(sorted({max(32, -(-int(nv_max) // (nsm * k))) for k in blocks_per_sm}))


FORM_NAMES = {S.SESW_FORM_AUTO: "", S.SESW_FORM_REGISTERS: " registers", S.SESW_FORM_STREAM: " streamed",
              S.SESW_FORM_STREAM_UNCACHED: " streamed-uncached"}


@dataclasses.dataclass
class Choice:
    mode: int
    blocks_per_sm: int = 0
    patch_vertices: int = 256
    block_threads: int = 256
    ms_per_step: float = float("inf")
    form: int = S.SESW_FORM_AUTO
    large_bps: int = 0          # batches: blocks per SM of the large basins' packs (0: blocks_per_sm)
    large_form: int = -1        # batches: their kernel form (-1: form)

    def apply(self, sim):
        sim.sesw_set_mode(self.mode)
        sim.sesw_set_blocks_per_sm(self.blocks_per_sm)
        sim.sesw_set_patch_vertices(self.patch_vertices)
        sim.sesw_set_block_threads(self.block_threads)
        sim.sesw_set_persistent_form(self.form)
        sim.sesw_set_large_basins(self.large_bps, self.large_form)

    def label(self):
        if self.mode == S.SESW_MODE_PERSISTENT:
            lab = f"persistent bps={self.blocks_per_sm}{FORM_NAMES[self.form]}"
            if self.large_bps or self.large_form >= 0:
                lf = self.form if self.large_form < 0 else self.large_form
                lab += f" large bps={self.large_bps or self.blocks_per_sm}{FORM_NAMES[lf]}"
            return lab
        return f"graph pv={self.patch_vertices} bt={self.block_threads}"


def _time_steps(sim, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        sim.sesw_advance(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        sim.sesw_advance(1)
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def autotune(meshes, params, forcing=None, steps=5, warmup=2, device=0, include_graph=True, include_persistent=True,
             graph_patches=GRAPH_PATCHES, graph_threads=GRAPH_THREADS, verbose=False,
             persistent_forms=(S.SESW_FORM_AUTO, S.SESW_FORM_STREAM), wave_sizes=True,
             large_layouts=((2, S.SESW_FORM_AUTO), (2, S.SESW_FORM_STREAM), (4, S.SESW_FORM_STREAM))):
    """Time every candidate layout on the meshes (a list: one mesh, or the basins of a batch).

    params: one Params per mesh. forcing: optional concatenated [sum E][2] array.
    Persistent candidates: every blocks-per-SM count with every kernel form of persistent_forms;
    for a batch also one block per SM for the common basins with each (blocks per SM, form) of
    large_layouts for the large ones.
    Graph candidates: graph_patches (plus, with wave_sizes, the one-wave patch sizes) with every
    block size of graph_threads.
    Returns (best Choice, list of (Choice, ms_per_step or None)).
    """
    import torch

    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    nv = sum(m.nv for m in meshes)
    ne = sum(m.ne for m in meshes)
    eta0 = np.zeros(nv)
    U0 = np.zeros((ne, 2))
    table = []

    def run(choice):
        with S.Subcycle(device, stream=stream) as sim:
            choice.apply(sim)
            if len(meshes) == 1:
                sim.sesw_mesh_upload(meshes[0])
                sim.sesw_set_params(params[0])
            else:
                sim.sesw_mesh_upload_batch(meshes)
                sim.sesw_set_params_batch(params)
            info = sim.sesw_get_info()
            if choice.mode == S.SESW_MODE_PERSISTENT and info["mode"] != S.SESW_MODE_PERSISTENT:
                return None
            if forcing is not None:
                sim.sesw_set_forcing(forcing)
            sim.sesw_set_state(eta0, U0)
            if choice.mode == S.SESW_MODE_GRAPH:
                # one upload serves every block size of this patch size
                out = []
                for bt in graph_threads:
                    sim.sesw_set_block_threads(bt)
                    out.append((bt, _time_steps(sim, steps, warmup, stream)))
                return out
            return _time_steps(sim, steps, warmup, stream)

    if include_persistent:
        cands = [Choice(S.SESW_MODE_PERSISTENT, blocks_per_sm=k, form=form)
                 for k in PERSISTENT_BLOCKS for form in persistent_forms]
        if len(meshes) > 1:
            cands += [Choice(S.SESW_MODE_PERSISTENT, blocks_per_sm=1, large_bps=lb, large_form=lf)
                      for lb, lf in large_layouts]
        for c in cands:
            try:
                t = run(c)
            except S.SeswError:
                t = None
            c.ms_per_step = t if t is not None else float("inf")
            table.append((c, t))
            if verbose:
                print(c.label(), t)
    if include_graph:
        nsm = torch.cuda.get_device_properties(device).multi_processor_count
        waves = set(wave_patch_sizes(max(m.nv for m in meshes), nsm)) if wave_sizes else set()
        patches = tuple(sorted(set(graph_patches) | waves))
        for pv in patches:
            try:
                res = run(Choice(S.SESW_MODE_GRAPH, patch_vertices=pv))
            except S.SeswError:
                res = None
            for bt in graph_threads:
                t = dict(res).get(bt) if res else None
                c = Choice(S.SESW_MODE_GRAPH, patch_vertices=pv, block_threads=bt,
                           ms_per_step=t if t is not None else float("inf"))
                table.append((c, t))
                if verbose:
                    print(c.label(), t)
    best = min((c for c, t in table if t is not None), key=lambda c: c.ms_per_step, default=None)
    if best is None:
        raise RuntimeError("no candidate layout ran on this mesh")
    return best, table
