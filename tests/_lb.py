"""Test helpers that move populations between the oracle's layout (Q, cells), in the oracle's
velocity order, and libsmrt states (library velocity order, padded planes, deviations
df_i = f_i - w_i with the library's own weights)."""
import numpy as np


def lib_from_oracle(olat, ldesc):
    """idx[i_lib] = i_oracle with equal integer velocity vectors."""
    key = {tuple(int(v) for v in e): i for i, e in enumerate(olat.e)}
    idx = np.array([key[tuple(int(v) for v in e)] for e in ldesc.e])
    assert sorted(idx.tolist()) == list(range(olat.q))
    return idx


def upload(ctx, f_oracle, idx):
    import torch
    st = ctx.new_state()
    flat = np.asarray(f_oracle).reshape(f_oracle.shape[0], -1)
    dev = flat[idx] - ctx.weights[:, None]
    ctx.planes(st)[:] = torch.from_numpy(np.ascontiguousarray(dev)).to(ctx.device, ctx.dtype)
    return st


def download(ctx, st, idx):
    arr = ctx.planes(st).double().cpu().numpy() + ctx.weights[:, None]
    out = np.empty_like(arr)
    out[idx] = arr
    return out
