"""Training and evaluation driver of the learned surrogate (the kernels are in the library).

The plain subcycle produces the training data: trajectories from rest under seeded
random forcing, each step recorded as (state, forcing) -> (increments of <<U>>, U^M and
the step-mean elevation). The network trains on the GPU with the library's Adam
kernels. Evaluation compares, on held-out trajectories, the surrogate against the
plain subcycle (the reference), against persistence (zero increments), and against
the plain subcycle with fewer substeps.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import inputs as I
from . import sesw as S


@dataclasses.dataclass
class Split:
    train: np.ndarray
    test: np.ndarray
    traj_len: int
    ntraj: int


def generate(sim, mesh, forcing_fn, ntraj, steps_per_traj, first_index=0):
    """Record ntraj trajectories of steps_per_traj steps from rest; sample k*steps_per_traj + n is
    step n of trajectory k. forcing_fn(k) returns the [E][2] forcing of trajectory k."""
    sim.sesw_set_eta_mean(True)
    zeta, zU = np.zeros(mesh.nv), np.zeros((mesh.ne, 2))
    i = first_index
    for k in range(ntraj):
        sim.sesw_set_forcing(forcing_fn(k))
        sim.sesw_set_state(zeta, zU)
        for _ in range(steps_per_traj):
            sim.sesw_surrogate_record_input(i)
            sim.sesw_advance(1)
            sim.sesw_surrogate_record_target(i)
            i += 1
    sim.sesw_set_eta_mean(False)
    if sim.sesw_status() != S.SESW_OK:
        raise RuntimeError("the plain subcycle flagged a device status while generating data")
    return i


def split(ntraj, steps_per_traj, test_fraction=0.1):
    ntest = max(1, int(round(ntraj * test_fraction)))
    idx = np.arange(ntraj * steps_per_traj).reshape(ntraj, steps_per_traj)
    return Split(idx[: ntraj - ntest].reshape(-1), idx[ntraj - ntest:].reshape(-1), steps_per_traj, ntraj)


def train(sim, train_idx, epochs, lr=2e-3, seed=0, lr_min_frac=0.05, log=None):
    """Per-sample Adam steps over shuffled epochs with a cosine learning-rate decay."""
    rng = np.random.default_rng(seed)
    total = epochs * len(train_idx)
    done = 0
    hist = []
    for ep in range(epochs):
        order = rng.permutation(train_idx)
        chunk = 64
        losses = []
        for c0 in range(0, len(order), chunk):
            frac = done / max(1, total)
            rate = lr * (lr_min_frac + (1 - lr_min_frac) * 0.5 * (1 + math.cos(math.pi * frac)))
            batch = order[c0:c0 + chunk]
            losses.append(sim.sesw_surrogate_train(batch, rate) * len(batch))
            done += len(batch)
        hist.append(sum(losses) / len(order))
        if log:
            log(f"epoch {ep}: mean train loss {hist[-1]:.4f}")
    return hist


def persistence_loss(sim, idx):
    """Loss of the all-zero prediction (what the method without the network predicts for the increments)."""
    w = sim.sesw_surrogate_weights()
    sim.sesw_surrogate_weights(set=np.zeros_like(w))
    try:
        return sim.sesw_surrogate_loss(idx)
    finally:
        sim.sesw_surrogate_weights(set=w)


SURROGATE_STEP_KERNELS = 15


def rollout_error(case, R, params_ref, weights, scales, nsteps, resid_tol, coarse_M=(), device=0,
                  surrogate_capacity=1):
    """From rest under forcing R: max |eta| difference to the plain subcycle after nsteps for the
    surrogate (with its fallback) and for the plain subcycle with fewer substeps; time per step."""
    import torch

    out = {}

    def plain(M):
        p = dataclasses.replace(params_ref, M=M)
        with S.Subcycle(device) as s:
            s.sesw_mesh_upload(case.mesh)
            s.sesw_set_params(p)
            s.sesw_set_forcing(R)
            s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
            s.sesw_advance(1)
            s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.sesw_advance(nsteps)
            eta = s.sesw_get_state()[0]
            return eta, (time.perf_counter() - t0) / nsteps

    ref, t_ref = plain(params_ref.M)
    out["plain"] = {"M": params_ref.M, "ms_per_step": 1e3 * t_ref, "max_ssh_error_m": 0.0}
    for M in coarse_M:
        try:
            eta, t = plain(M)
            out[f"plain_M{M}"] = {"M": M, "ms_per_step": 1e3 * t,
                                  "max_ssh_error_m": float(np.max(np.abs(eta - ref)))}
        except S.SeswError as e:
            out[f"plain_M{M}"] = {"M": M, "rejected": str(e)}
    with S.Subcycle(device) as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(params_ref)
        s.sesw_surrogate_init(surrogate_capacity, seed=0)
        s.sesw_surrogate_weights(set=weights)
        s.sesw_surrogate_scales(set=scales)
        s.sesw_set_forcing(R)
        s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
        info = s.sesw_get_info()
        s.sesw_surrogate_advance(1, resid_tol)
        s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nfb, resid = s.sesw_surrogate_advance(nsteps, resid_tol)
        eta = s.sesw_get_state()[0]
        t = (time.perf_counter() - t0) / nsteps
        # the same without fallback: what the network alone does
        s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
        t1 = time.perf_counter()
        _, resid_nofb = s.sesw_surrogate_advance(nsteps, 1e30)
        eta_nofb = s.sesw_get_state()[0]
        t_nofb = (time.perf_counter() - t1) / nsteps
    # kernels per surrogate step: state copy-in, features, 10 of the forward pass, apply to
    # elements and vertices, residual; a fallback adds one plain step (one cooperative launch
    # per pack, or M substeps and the epilogue in graph mode)
    plain_launches = max(1, info["npack"]) if info["mode"] == S.SESW_MODE_PERSISTENT else params_ref.M + 1
    out["surrogate"] = {"resid_tol": resid_tol, "fallback_steps": nfb, "steps": nsteps,
                        "ms_per_step": 1e3 * t, "max_ssh_error_m": float(np.max(np.abs(eta - ref))),
                        "last_residual": resid, "gpu_launches": nsteps * SURROGATE_STEP_KERNELS + nfb * plain_launches}
    out["surrogate_no_fallback"] = {"ms_per_step": 1e3 * t_nofb,
                                    "max_ssh_error_m": float(np.max(np.abs(eta_nofb - ref))),
                                    "last_residual": resid_nofb}
    out["max_ssh_reference_m"] = float(np.max(np.abs(ref)))
    return out


def gain_summary(roll):
    """What each cheaper form gains over the plain subcycle at M: its speedup (plain time per step
    over its own) and the SSH error it pays for it, from a rollout_error result."""
    plain_ms = roll["plain"]["ms_per_step"]
    out = {}
    for name, r in roll.items():
        if name == "plain" or not isinstance(r, dict) or "ms_per_step" not in r:
            continue
        out[name] = {"speedup_vs_plain": plain_ms / r["ms_per_step"], "max_ssh_error_m": r["max_ssh_error_m"],
                     "ms_per_step": r["ms_per_step"]}
    return out


def sphere_forcing(case, seed):
    """Smooth random forcing of the sphere workload (new seed per trajectory)."""
    H0e = case.mesh.depth[case.mesh.tri].mean(axis=1)
    a = I.smooth_element_field(case.mesh.pos, case.mesh.tri, seed, amp=1e-6)
    return H0e[:, None] * a
