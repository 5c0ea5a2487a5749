"""FP64 numpy reference of the message-passing surrogate (forward and analytic backward).

TEST INFRASTRUCTURE ONLY (see the package docstring). The paper has no surrogate; this
module defines the network the library's CUDA kernels implement, written plainly:

Scales s = (eta, H, U, R, f, L, out_U, out_eta); hidden width C = 64; layers = 3.
Vertex inputs  x_v = [eta/s_eta, H0/s_H]; element inputs x_e = [U/s_U (2), R/s_R (2),
f/s_f, H0_e/s_H], with H0_e the corner mean of H0.

    h_v = tanh(x_v Wv0 + bv0),  h_e = tanh(x_e We0 + be0)
    for l in 1..3:
        z_e = [h_e, L sum_k dphi_k/dx h_{v_k}, L sum_k dphi_k/dy h_{v_k}]      (192)
        h_e = h_e + tanh(z_e We_l + be_l)
        z_v = [h_v, sum_{e ni v} A_e h_e / sum_{e ni v} A_e]                 (128)
        h_v = h_v + tanh(z_v Wv_l + bv_l)
    o_e = h_e Weo + beo (4),  o_v = h_v Wvo + bvo (1)

With bf16_msgs (the GPU's form) the concatenated inputs z_e and z_v of the message layers are
rounded to bfloat16 values when they are formed: the layers run on BF16 tensor-core operands.
The backward then passes gradients through the rounding unchanged, and the weight gradients
use the rounded inputs.

Predicted one-step increments: <<U>> - U = s_out_U o_e[0:2], U^M - U = s_out_U o_e[2:4],
eta_bar - eta = s_out_eta o_v. Loss: mean over elements and channels of (o_e - t_e)^2
plus mean over vertices of (o_v - t_v)^2 (t: targets divided by their scales).
Parameters are one flat vector in the order of ``param_shapes``; matrices are K x C,
row-major.
"""
from __future__ import annotations

import numpy as np

C = 64
LAYERS = 3


def param_shapes():
    shapes = [("Wv0", (2, C)), ("bv0", (C,)), ("We0", (6, C)), ("be0", (C,))]
    for l in range(1, LAYERS + 1):
        shapes += [(f"We{l}", (3 * C, C)), (f"be{l}", (C,)), (f"Wv{l}", (2 * C, C)), (f"bv{l}", (C,))]
    shapes += [("Weo", (C, 4)), ("beo", (4,)), ("Wvo", (C, 1)), ("bvo", (1,))]
    return shapes


def unflatten(w):
    out, o = {}, 0
    for name, shp in param_shapes():
        n = int(np.prod(shp))
        out[name] = w[o:o + n].reshape(shp)
        o += n
    assert o == len(w)
    return out


def nparams():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even) and return float64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def quantise(w):
    """Matrices rounded to bfloat16 as the GPU uses them; biases kept."""
    p = unflatten(np.asarray(w, dtype=np.float64).copy())
    for name, _ in param_shapes():
        if name.startswith("W"):
            p[name][...] = bf16_round(p[name])
    return np.concatenate([p[n].reshape(-1) for n, _ in param_shapes()])


class Graph:
    """Mesh geometry for the network: P1 gradients, areas, vertex incidence (own code)."""

    def __init__(self, mesh):
        xy = np.asarray(mesh.xy, dtype=np.float64)
        self.tri = np.asarray(mesh.tri, dtype=np.int64)
        self.nv, self.ne = int(mesh.nv), int(mesh.tri.shape[0])
        p0, p1, p2 = xy[:, 0], xy[:, 1], xy[:, 2]
        self.area = 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))
        self.grad = np.zeros((self.ne, 3, 2))
        for k in range(3):
            d = xy[:, (k + 2) % 3] - xy[:, (k + 1) % 3]
            self.grad[:, k, 0] = -d[:, 1] / (2 * self.area)
            self.grad[:, k, 1] = d[:, 0] / (2 * self.area)
        self.asum = np.zeros(self.nv)
        for k in range(3):
            np.add.at(self.asum, self.tri[:, k], self.area)
        self.H0v = np.asarray(mesh.depth, dtype=np.float64)
        self.H0e = self.H0v[self.tri].mean(axis=1)
        self.f = np.asarray(mesh.coriolis, dtype=np.float64)

    def grad_msg(self, hv, L):
        gx = np.zeros((self.ne, hv.shape[1]))
        gy = np.zeros((self.ne, hv.shape[1]))
        for k in range(3):
            gx += self.grad[:, k, 0:1] * hv[self.tri[:, k]]
            gy += self.grad[:, k, 1:2] * hv[self.tri[:, k]]
        return L * gx, L * gy

    def grad_msg_adj(self, dgx, dgy, L):
        dhv = np.zeros((self.nv, dgx.shape[1]))
        for k in range(3):
            np.add.at(dhv, self.tri[:, k], L * (self.grad[:, k, 0:1] * dgx + self.grad[:, k, 1:2] * dgy))
        return dhv

    def mean_msg(self, he):
        m = np.zeros((self.nv, he.shape[1]))
        for k in range(3):
            np.add.at(m, self.tri[:, k], self.area[:, None] * he)
        return m / self.asum[:, None]

    def mean_msg_adj(self, dm):
        dhe = np.zeros((self.ne, dm.shape[1]))
        for k in range(3):
            dhe += self.area[:, None] * (dm[self.tri[:, k]] / self.asum[self.tri[:, k], None])
        return dhe


def features(G, eta, U, R, s):
    xv = np.stack([eta / s["eta"], G.H0v / s["H"]], axis=1)
    xe = np.concatenate([U / s["U"], R / s["R"], (G.f / s["f"])[:, None], (G.H0e / s["H"])[:, None]], axis=1)
    return xv, xe


def forward(G, w, xv, xe, s, keep=False, bf16_msgs=False):
    p = unflatten(w)
    q = bf16_round if bf16_msgs else (lambda x: x)
    hv = np.tanh(xv @ p["Wv0"] + p["bv0"])
    he = np.tanh(xe @ p["We0"] + p["be0"])
    cache = {"hv": [hv], "he": [he], "ye": [], "yv": [], "ze": [], "zv": []}
    for l in range(1, LAYERS + 1):
        gx, gy = G.grad_msg(hv, s["L"])
        ze = q(np.concatenate([he, gx, gy], axis=1))
        ye = np.tanh(ze @ p[f"We{l}"] + p[f"be{l}"])
        he = he + ye
        zv = q(np.concatenate([hv, G.mean_msg(he)], axis=1))
        yv = np.tanh(zv @ p[f"Wv{l}"] + p[f"bv{l}"])
        hv = hv + yv
        if keep:
            cache["ze"].append(ze)
            cache["zv"].append(zv)
            cache["ye"].append(ye)
            cache["yv"].append(yv)
            cache["hv"].append(hv)
            cache["he"].append(he)
    oe = he @ p["Weo"] + p["beo"]
    ov = hv @ p["Wvo"] + p["bvo"]
    return (oe, ov, cache) if keep else (oe, ov)


def loss(oe, ov, te, tv):
    return float(np.mean((oe - te) ** 2) + np.mean((ov - tv) ** 2))


def loss_and_grad(G, w, xv, xe, te, tv, s, bf16_msgs=False):
    """Loss and its gradient with respect to the flat parameter vector (analytic backward)."""
    p = unflatten(w)
    oe, ov, c = forward(G, w, xv, xe, s, keep=True, bf16_msgs=bf16_msgs)
    L = loss(oe, ov, te, tv)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    doe = 2.0 * (oe - te) / oe.size
    dov = 2.0 * (ov - tv) / ov.size
    he, hv = c["he"][-1], c["hv"][-1]
    g["Weo"] = he.T @ doe
    g["beo"] = doe.sum(axis=0)
    g["Wvo"] = hv.T @ dov
    g["bvo"] = dov.sum(axis=0)
    dhe = doe @ p["Weo"].T
    dhv = dov @ p["Wvo"].T
    for l in range(LAYERS, 0, -1):
        # vertex update of layer l
        da = dhv * (1 - c["yv"][l - 1] ** 2)
        g[f"Wv{l}"] = c["zv"][l - 1].T @ da
        g[f"bv{l}"] = da.sum(axis=0)
        dz = da @ p[f"Wv{l}"].T
        dhv = dhv + dz[:, :C]
        dhe = dhe + G.mean_msg_adj(dz[:, C:])
        # element update of layer l
        da = dhe * (1 - c["ye"][l - 1] ** 2)
        g[f"We{l}"] = c["ze"][l - 1].T @ da
        g[f"be{l}"] = da.sum(axis=0)
        dz = da @ p[f"We{l}"].T
        dhe = dhe + dz[:, :C]
        dhv = dhv + G.grad_msg_adj(dz[:, C:2 * C], dz[:, 2 * C:], s["L"])
    da = dhv * (1 - c["hv"][0] ** 2)
    g["Wv0"] = xv.T @ da
    g["bv0"] = da.sum(axis=0)
    da = dhe * (1 - c["he"][0] ** 2)
    g["We0"] = xe.T @ da
    g["be0"] = da.sum(axis=0)
    return L, np.concatenate([g[n].reshape(-1) for n, _ in param_shapes()])
