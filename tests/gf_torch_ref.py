"""Independent restatement of the graph-family energy in PyTorch FP64 (test-only).

Edges from the numpy brute-force neighbour selection of ``af_torch_ref``; the
node/edge/angle stack as dense tensor ops over padded edge arrays; forces by
torch.autograd.  Agreement with the C oracle pins the oracle's hand-written
backward and bookkeeping to a second reading of the same model.
"""
from __future__ import annotations

import numpy as np
import torch

from tests.af_torch_ref import select_neighbours


def parse_blob(d: dict, blob):
    w = torch.as_tensor(np.asarray(blob, dtype=np.float64))
    pos = 0

    def take(*shape):
        nonlocal pos
        n = int(np.prod(shape))
        t = w[pos:pos + n].reshape(*shape)
        pos += n
        return t

    Nd, Ed, S = d["node"], d["edge"], d["n_species"]
    g = dict(Wt=take(S, Nd), we=take(Ed), be0=take(Ed))
    layers = [dict(Wm=take(Nd, Ed), Wn=take(Nd + Ed, Nd), bn=take(Nd), Wa=take(Nd, Ed),
                   Wb=take(Nd, Ed), Wc=take(Ed, Ed), be=take(Ed), Wp=take(Ed, Ed), Wphi=take(4, Ed),
                   Wq=take(Ed, Ed), bq=take(Ed)) for _ in range(d["n_layers"])]
    fit = [dict(F1=take(Nd, d["f1"]), c1=take(d["f1"]), F2=take(d["f1"], d["f2"]), c2=take(d["f2"]),
                F3=take(d["f2"], d["f3"]), c3=take(d["f3"]), F4=take(d["f3"], 1), c4=take(1))
           for _ in range(S)]
    assert pos == len(w)
    return g, layers, fit


def switch(r, rs, rc):
    u = (r - rs) / (rc - rs)
    poly = u ** 3 * (-6 * u ** 2 + 15 * u - 10) + 1
    return torch.where(r < rs, torch.ones_like(r), torch.where(r < rc, poly, torch.zeros_like(r)))


def energy(d: dict, blob, types, coords, box):
    g, layers, fit = parse_blob(d, blob)
    types = np.asarray(types)
    n = len(types)
    NM, NA = d["nmax"], d["na"]
    L = torch.as_tensor(np.asarray(box, dtype=np.float64))
    nb = select_neighbours(coords.detach().numpy(), box, d["rc"], NM)
    cnt = np.array([len(r) for r in nb])
    J = np.zeros((n, NM), dtype=np.int64)
    IMG = np.zeros((n, NM, 3))
    mask = np.zeros((n, NM), dtype=bool)
    for i, row in enumerate(nb):
        for p, (j, im) in enumerate(row):
            J[i, p], IMG[i, p], mask[i, p] = j, im, True
    J = torch.as_tensor(J)
    M = torch.as_tensor(mask, dtype=torch.float64)
    x = coords
    wrap = torch.floor(x.detach() / L)
    r = x[J] - x[:, None, :] + (torch.as_tensor(IMG) - wrap[J] + wrap[:, None, :]) * L
    r = torch.where(M[..., None] > 0, r, torch.ones_like(r))      # keep padding finite
    dist = torch.sqrt((r * r).sum(-1))
    sw = switch(dist, d["rs"], d["rc"]) * M
    s = sw / dist
    rh = r / dist[..., None]
    # angle slots: the first (nearest) slots with r < rca, at most na
    amask = (dist < d["rca"]) & (M > 0)
    amask = amask & (torch.cumsum(amask.to(torch.int64), 1) <= NA)
    A = amask.to(torch.float64)
    swa = switch(dist, d["rsa"], d["rca"]) * A
    cos = torch.einsum("ipa,ika->ipk", rh, rh)
    P = torch.stack([torch.ones_like(cos), cos, 0.5 * (3 * cos ** 2 - 1),
                     0.5 * (5 * cos ** 3 - 3 * cos)])                # (4, n, p, k)
    offdiag = 1.0 - torch.eye(NM, dtype=torch.float64)
    pair = swa[:, :, None] * swa[:, None, :] * offdiag / NA          # (n, p, k)
    nodes = g["Wt"][torch.as_tensor(types)]
    e = torch.tanh(s[..., None] * g["we"] + g["be0"]) * M[..., None]
    for lw in layers:
        u = nodes @ lw["Wm"]
        m = (sw[..., None] * e * u[J]).sum(1) / NM
        nodes = nodes + torch.tanh(torch.cat([nodes, m], 1) @ lw["Wn"] + lw["bn"])
        v = torch.tanh((nodes @ lw["Wa"])[:, None, :] + (nodes @ lw["Wb"])[J] + e @ lw["Wc"] + lw["be"])
        e = (e + v) * M[..., None]
        q = e @ lw["Wp"]
        a = torch.einsum("lc,lipk,ipk,ikc->ipc", lw["Wphi"], P, pair, q)
        e = e + swa[..., None] * torch.tanh(a @ lw["Wq"] + lw["bq"])
    E = torch.zeros((), dtype=torch.float64)
    for i in range(n):
        f = fit[int(types[i])]
        y = torch.tanh(nodes[i] @ f["F1"] + f["c1"])
        y = torch.tanh(y @ f["F2"] + f["c2"])
        y = torch.tanh(y @ f["F3"] + f["c3"])
        E = E + (y @ f["F4"] + f["c4"])[0]
    del cnt
    return E
