"""Independent restatement of the attention-family energy in PyTorch FP64.

Test-only.  Written separately from the C oracle: neighbours by numpy brute
force over images, the network as batched tensor ops, and the gradient by
torch.autograd instead of a hand-derived adjoint.  Agreement with the oracle
pins the oracle's backward pass and its bookkeeping (weight blob order,
neighbour selection, normalisations) to a second reading of the same model.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch


def parse_blob(model: dict, blob: np.ndarray):
    """Split the blob in its documented order into named tensors."""
    d = model
    w = torch.as_tensor(np.asarray(blob, dtype=np.float64))
    pos = 0

    def take(*shape):
        nonlocal pos
        n = int(np.prod(shape))
        t = w[pos:pos + n].reshape(*shape)
        pos += n
        return t

    S, L = d["n_species"], d["n_layers"]
    emb = [dict(W1=take(1, d["e1"]), b1=take(d["e1"]), W2=take(d["e1"], d["e2"]), b2=take(d["e2"]),
                W3=take(d["e2"], d["m1"]), b3=take(d["m1"])) for _ in range(S)]
    att = [dict(Wq=take(d["m1"], d["hidden"]), Wk=take(d["m1"], d["hidden"]),
                Wv=take(d["m1"], d["hidden"]), Wo=take(d["hidden"], d["m1"]), bo=take(d["m1"]))
           for _ in range(L)]
    fit = [dict(W1=take(d["m1"] * d["m2"], d["f1"]), b1=take(d["f1"]), W2=take(d["f1"], d["f2"]),
                b2=take(d["f2"]), W3=take(d["f2"], d["f3"]), b3=take(d["f3"]), W4=take(d["f3"], 1),
                b4=take(1)) for _ in range(S)]
    assert pos == len(w), (pos, len(w))
    return emb, att, fit


def select_neighbours(coords, box, rc, nmax):
    """numpy brute force: per atom, the nmax nearest (j, image) with 0 < r < rc,
    ordered by (r^2, j, image)."""
    x = np.asarray(coords, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    w = x - L * np.floor(x / L)
    n = len(x)
    nimg = [int(math.ceil(rc / L[a])) + 1 for a in range(3)]
    imgs = np.array(list(itertools.product(*[range(-k, k + 1) for k in nimg])), dtype=np.int64)
    out = []
    for i in range(n):
        r = (w[None, :, :] - w[i][None, None, :]) + imgs[:, None, :] * L[None, None, :]
        d2 = (r[..., 0] * r[..., 0] + r[..., 1] * r[..., 1]) + r[..., 2] * r[..., 2]
        ii, jj = np.nonzero((d2 < rc * rc) & (d2 > 0))
        keys = [(d2[a, b], int(jj[k]), tuple(int(v) for v in imgs[a]))
                for k, (a, b) in enumerate(zip(ii, jj))]
        keys.sort()
        out.append([(j, np.array(img)) for _, j, img in keys[:nmax]])
    return out


def switch(r, rs, rc):
    u = (r - rs) / (rc - rs)
    poly = u ** 3 * (-6 * u ** 2 + 15 * u - 10) + 1
    return torch.where(r < rs, torch.ones_like(r), torch.where(r < rc, poly, torch.zeros_like(r)))


def energy(model: dict, blob, types, coords, box, nbrs=None):
    """E (torch scalar) with autograd through ``coords`` (a leaf tensor)."""
    d = model
    emb, att, fit = parse_blob(d, blob)
    x = coords
    L = torch.as_tensor(np.asarray(box, dtype=np.float64))
    if nbrs is None:
        nbrs = select_neighbours(x.detach().numpy(), box, d["rc"], d["nmax"])
    types = np.asarray(types)
    nh, H = d["heads"], d["hidden"]
    dh = H // nh
    E = torch.zeros((), dtype=torch.float64)
    for i in range(len(types)):
        lst = nbrs[i]
        if lst:
            js = torch.as_tensor([j for j, _ in lst])
            imgs = torch.as_tensor(np.stack([im for _, im in lst]), dtype=torch.float64)
            # wrapping only shifts by whole box lengths: fold it into the image
            wrap_i = torch.floor(x[i].detach() / L)
            wrap_j = torch.floor(x[js].detach() / L)
            r = x[js] - x[i] + (imgs - wrap_j + wrap_i) * L
            dist = torch.sqrt((r * r).sum(-1))
            sw = switch(dist, d["rs"], d["rc"])
            s = sw / dist
            rhat = r / dist[:, None]
            Rt = torch.cat([s[:, None], s[:, None] * rhat], 1)           # (n, 4)
            tj = types[js.numpy()]
            G = torch.stack([
                torch.tanh(torch.tanh(torch.tanh(s[k:k + 1] @ emb[t]["W1"] + emb[t]["b1"])
                                      @ emb[t]["W2"] + emb[t]["b2"]) @ emb[t]["W3"] + emb[t]["b3"])
                for k, t in enumerate(tj)])                               # (n, m1)
            gate = rhat @ rhat.T
            for lw in att:
                q = (G @ lw["Wq"]).reshape(-1, nh, dh).transpose(0, 1)   # (nh, n, dh)
                k = (G @ lw["Wk"]).reshape(-1, nh, dh).transpose(0, 1)
                v = (G @ lw["Wv"]).reshape(-1, nh, dh).transpose(0, 1)
                sc = q @ k.transpose(1, 2) / math.sqrt(dh)
                wts = sw[None, None, :] * torch.exp(sc - sc.max(-1, keepdim=True).values.detach())
                wts = wts / wts.sum(-1, keepdim=True)
                o = (wts * gate[None]) @ v                                # (nh, n, dh)
                o = o.transpose(0, 1).reshape(-1, H)
                z = G + o @ lw["Wo"] + lw["bo"]
                G = torch.nn.functional.layer_norm(z, (d["m1"],), eps=1e-5)
            T = Rt.T @ G / d["nmax"]                                      # (4, m1)
            D = (T.T @ T[:, :d["m2"]]).reshape(-1)
        else:
            D = torch.zeros(d["m1"] * d["m2"], dtype=torch.float64)
        f = fit[int(types[i])]
        y = torch.tanh(D @ f["W1"] + f["b1"])
        y = torch.tanh(y @ f["W2"] + f["b2"])
        y = torch.tanh(y @ f["W3"] + f["b3"])
        E = E + (y @ f["W4"] + f["b4"])[0]
    return E


def parse_blob_mp(model: dict, blob: np.ndarray):
    """Message-passing blob: embedding nets, the atom channel's species rows
    Wt, per layer the attention weights then Wm and bm, fitting nets."""
    d = model
    w = torch.as_tensor(np.asarray(blob, dtype=np.float64))
    pos = 0

    def take(*shape):
        nonlocal pos
        n = int(np.prod(shape))
        t = w[pos:pos + n].reshape(*shape)
        pos += n
        return t

    S, L, M1 = d["n_species"], d["n_layers"], d["m1"]
    emb = [dict(W1=take(1, d["e1"]), b1=take(d["e1"]), W2=take(d["e1"], d["e2"]), b2=take(d["e2"]),
                W3=take(d["e2"], M1), b3=take(M1)) for _ in range(S)]
    Wt = take(S, M1)
    att = [dict(Wq=take(M1, d["hidden"]), Wk=take(M1, d["hidden"]), Wv=take(M1, d["hidden"]),
                Wo=take(d["hidden"], M1), bo=take(M1), Wm=take(M1, M1), bm=take(M1))
           for _ in range(L)]
    fit = [dict(W1=take(M1 * d["m2"], d["f1"]), b1=take(d["f1"]), W2=take(d["f1"], d["f2"]),
                b2=take(d["f2"]), W3=take(d["f2"], d["f3"]), b3=take(d["f3"]), W4=take(d["f3"], 1),
                b4=take(1)) for _ in range(S)]
    assert pos == len(w), (pos, len(w))
    return emb, Wt, att, fit


def energy_mp(model: dict, blob, types, coords, box, nbrs=None):
    """E with an atom channel passed between neighbours (autograd through
    ``coords``): h^0 = Wt[t]; per layer U = tanh(h Wm + bm), every kept slot's
    pair feature gains its neighbour's U before the attention layer, and
    h += (1/Nmax) sum_p sw_p G_p of the layer's output (not after the last)."""
    d = model
    emb, Wt, att, fit = parse_blob_mp(d, blob)
    x = coords
    Lb = torch.as_tensor(np.asarray(box, dtype=np.float64))
    if nbrs is None:
        nbrs = select_neighbours(x.detach().numpy(), box, d["rc"], d["nmax"])
    types = np.asarray(types)
    n, nh, H, M1 = len(types), d["heads"], d["hidden"], d["m1"]
    dh = H // nh
    env = []
    for i in range(n):
        lst = nbrs[i]
        if not lst:
            env.append(None)
            continue
        js = torch.as_tensor([j for j, _ in lst])
        imgs = torch.as_tensor(np.stack([im for _, im in lst]), dtype=torch.float64)
        wrap_i = torch.floor(x[i].detach() / Lb)
        wrap_j = torch.floor(x[js].detach() / Lb)
        r = x[js] - x[i] + (imgs - wrap_j + wrap_i) * Lb
        dist = torch.sqrt((r * r).sum(-1))
        sw = switch(dist, d["rs"], d["rc"])
        s = sw / dist
        rhat = r / dist[:, None]
        Rt = torch.cat([s[:, None], s[:, None] * rhat], 1)
        tj = types[js.numpy()]
        G = torch.stack([
            torch.tanh(torch.tanh(torch.tanh(s[k:k + 1] @ emb[t]["W1"] + emb[t]["b1"])
                                  @ emb[t]["W2"] + emb[t]["b2"]) @ emb[t]["W3"] + emb[t]["b3"])
            for k, t in enumerate(tj)])
        env.append(dict(js=js, sw=sw, Rt=Rt, gate=rhat @ rhat.T, G=G))
    h = Wt[torch.as_tensor(types, dtype=torch.long)]
    for l, lw in enumerate(att):
        U = torch.tanh(h @ lw["Wm"] + lw["bm"])
        pooled = []
        for i in range(n):
            e = env[i]
            if e is None:
                pooled.append(torch.zeros(M1, dtype=torch.float64))
                continue
            G = e["G"] + U[e["js"]]
            q = (G @ lw["Wq"]).reshape(-1, nh, dh).transpose(0, 1)
            k = (G @ lw["Wk"]).reshape(-1, nh, dh).transpose(0, 1)
            v = (G @ lw["Wv"]).reshape(-1, nh, dh).transpose(0, 1)
            sc = q @ k.transpose(1, 2) / math.sqrt(dh)
            wts = e["sw"][None, None, :] * torch.exp(sc - sc.max(-1, keepdim=True).values.detach())
            wts = wts / wts.sum(-1, keepdim=True)
            o = ((wts * e["gate"][None]) @ v).transpose(0, 1).reshape(-1, H)
            G = torch.nn.functional.layer_norm(G + o @ lw["Wo"] + lw["bo"], (M1,), eps=1e-5)
            e["G"] = G
            pooled.append((e["sw"][:, None] * G).sum(0) / d["nmax"])
        if l + 1 < len(att):
            h = h + torch.stack(pooled)
    E = torch.zeros((), dtype=torch.float64)
    for i in range(n):
        e = env[i]
        if e is None:
            D = torch.zeros(M1 * d["m2"], dtype=torch.float64)
        else:
            T = e["Rt"].T @ e["G"] / d["nmax"]
            D = (T.T @ T[:, :d["m2"]]).reshape(-1)
        f = fit[int(types[i])]
        y = torch.tanh(D @ f["W1"] + f["b1"])
        y = torch.tanh(y @ f["W2"] + f["b2"])
        y = torch.tanh(y @ f["W3"] + f["b3"])
        E = E + (y @ f["W4"] + f["b4"])[0]
    return E
