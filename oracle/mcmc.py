"""Oracle of the codebook sampler's transitions -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and bench.py's CPU legs may
import this module; the CUDA library never does.

The sampler of Secs. 4.3-4.4 and Appendix A.1 moves the state S = {G, C} by one of
three transitions:

* parameter update (SGLD, Sec. 2.3.2, Eq. 9, and Eqs. 25-28 of Appendix A.1): every differentiable
  tensor X in {positions, opacity logits, SR rows, SH rows} becomes
  X + (eps_X / 2) grad log p + sqrt(eps_X) eta with eta ~ N(0, I), where
  grad log p = -grad L (p proportional to exp(-L), Eq. 12);
* split (Sec. 4.4, Eqs. 16-17, 19): a Gaussian mapped to row c gets a new row c'' = c + u,
  u ~ N(0, eps_split^2 I), accepted with min(1, e^-lambda / q_sm(u));
* merge (Sec. 4.4, Eqs. 18, 20): a row c' split from c is merged back into c, proposed
  with the kernel N(c - c' | 0, eps_merge^2 I) and accepted with
  min(1, e^lambda q_sm(c - c')),
  with q_sm(u) = exp(-(|u|^2 / 2)(1 / eps_split^2 - 1 / eps_merge^2)).

Random draws come from Philox4x32-10 (Salmon et al., SC'11), a
counter-based generator that both this oracle and the kernels implement from
its published definition; normals are Box-Muller (1958) pairs.  Parameter
updates are continuous, so the oracle computes them in FP64 (normals from
FP64 Box-Muller of the same bits).  Split and merge outcomes are integers
decided by floating point, so the oracle takes them in FP32 with the written
operation order that the kernels follow (``mcmc32.c``), and the new rows are
FP32 sums c + u, i.e. exact binary32 results.

Counter layout (key = the 64-bit seed, low word first):
  c0 = element >> 2 (updates) / Gaussian (split) / row (merge),
  c1 = stream | call << 8, c2, c3 = low and high word of the step.
Streams: 0 positions, 1 opacity logits, 2 SR rows, 3 SH rows (updates);
16 + b split normals, 18 + b split acceptance, 20 + b merge draws, with
b = 0 for the SR codebook and 1 for the SH codebook.
"""
from __future__ import annotations

import numpy as np

from . import _ptr, lib

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_POS, STREAM_LOGIT, STREAM_SR, STREAM_SH = 0, 1, 2, 3
STREAM_SPLIT_U, STREAM_SPLIT_V, STREAM_MERGE = 16, 18, 20
SR_WIDTH = 8      # SR row: 3 log-scales, 4 quaternion values (w, x, y, z), 1 unused
SR_DIMS = 7       # values of an SR row that the sampler moves


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ctr: (..., 4) uint32, key: (..., 2)
    uint32 (broadcast).  One round maps (c0, c1, c2, c3) with key (k0, k1)
    to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key is advanced by the Weyl constants (W0, W1) before every round
    after the first."""
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = np.broadcast_to(k[..., 0], c0.shape), np.broadcast_to(k[..., 1], c0.shape)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & MASK32
            k1 = (k1 + np.uint64(W1)) & MASK32
        p0 = c0 * np.uint64(M0)
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def draws(index, stream: int, call: int, step: int, seed: int) -> np.ndarray:
    """Philox outputs for counters (index, stream | call << 8, step)."""
    idx = np.asarray(index, dtype=np.uint64).ravel()
    ctr = np.empty((idx.size, 4), dtype=np.uint64)
    ctr[:, 0] = idx & MASK32
    ctr[:, 1] = np.uint64(stream | (call << 8))
    ctr[:, 2] = np.uint64(step & 0xFFFFFFFF)
    ctr[:, 3] = np.uint64((step >> 32) & 0xFFFFFFFF)
    return philox4x32_10(ctr, seed_key(seed))


def normals64(bits: np.ndarray) -> np.ndarray:
    """FP64 Box-Muller: (count, 4) draws -> (count, 4) standard normals,
    pairs (0, 1) and (2, 3): u1 = ((a >> 8) + 1) 2^-24 in (0, 1],
    u2 = (b >> 8) 2^-24 in [0, 1), z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2)."""
    b = bits.astype(np.float64)
    a0 = np.floor(b[:, 0::2] / 256.0)
    a1 = np.floor(b[:, 1::2] / 256.0)
    u1 = (a0 + 1.0) * 2.0 ** -24
    u2 = a1 * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(b.shape, dtype=np.float64)
    out[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    out[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return out


def normals32(bits: np.ndarray) -> np.ndarray:
    """The same normals in the FP32 decision arithmetic (mcmc32.c)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    z = np.empty(bits.shape, dtype=np.float32)
    lib().or_normals32(bits.shape[0], _ptr(bits), _ptr(z))
    return z


def uniform32(a: np.ndarray) -> np.ndarray:
    """Uniform in [0, 1) from the top 24 bits of a draw (exact in FP32)."""
    return ((np.asarray(a, dtype=np.uint32) >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24))


def log32(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.empty_like(x)
    lib().or_log32_batch(x.size, _ptr(x), _ptr(y))
    return y


def sincos2pi32(u):
    u = np.ascontiguousarray(u, dtype=np.float32).ravel()
    s, c = np.empty_like(u), np.empty_like(u)
    lib().or_sincos2pi32_batch(u.size, _ptr(u), _ptr(s), _ptr(c))
    return s, c


def exp32(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.empty_like(x)
    lib().or_e32_batch(x.size, _ptr(x), _ptr(y))
    return y


def bf16_rne(x) -> np.ndarray:
    """binary32 -> bfloat16 (round to nearest even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (r.astype(np.uint32) << np.uint32(16)).view(np.float32)


def bf16_rne64(x) -> np.ndarray:
    """binary64 -> bfloat16 rounded once (nearest, ties to even), as float32:
    x = m 2^e with m in [0.5, 1), m 2^8 rounded to an integer (exact FP64
    operations), scaled back."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8).astype(np.float32)


# ----------------------------------------------------------------------------
# parameter update (SGLD)
# ----------------------------------------------------------------------------

def _sgld_tensor(x, g, eps, stream, step, seed, cols=None, width=None):
    """x + (eps/2)(-g) + sqrt(eps) z over the elements of one tensor, in
    FP64.  Element e draws normal e & 3 of call e >> 2.  With ``cols``,
    only those columns of rows of ``width`` values move."""
    x64 = np.asarray(x, dtype=np.float64).ravel()
    g64 = np.asarray(g, dtype=np.float64).ravel()
    m = x64.size
    calls = (m + 3) // 4
    z = normals64(draws(np.arange(calls), stream, 0, step, seed)).ravel()[:m]
    out = x64 + (eps / 2.0) * (-g64) + np.sqrt(eps) * z
    if cols is not None:
        moving = np.zeros(width, dtype=bool)
        moving[list(cols)] = True
        keep = ~np.tile(moving, m // width)
        out[keep] = x64[keep]
    return out.reshape(np.shape(x))


def sgld_update(scene, grads: dict, eps: dict, step: int, seed: int, bf16: bool = False) -> dict:
    """One parameter-update transition.  grads: dpos [N,3], dlogit [N],
    d_sr [K_sr,8], d_sh [K_sh,B,3] (gradients of the loss L); eps: step sizes
    'pos', 'logit', 'sr', 'sh'.  Returns FP64 tensors (SR / SH rows rounded
    once to BF16 when the codebooks are stored in BF16)."""
    out = {
        "pos": _sgld_tensor(scene.pos, grads["dpos"], eps["pos"], STREAM_POS, step, seed),
        "logit": _sgld_tensor(scene.opacity_logit, grads["dlogit"], eps["logit"], STREAM_LOGIT, step, seed),
        "sr": _sgld_tensor(scene.sr_rows, grads["d_sr"], eps["sr"], STREAM_SR, step, seed,
                           cols=range(SR_DIMS), width=SR_WIDTH),
        "sh": _sgld_tensor(scene.sh_rows, grads["d_sh"], eps["sh"], STREAM_SH, step, seed),
    }
    if bf16:
        out["sr"] = bf16_rne64(out["sr"]).astype(np.float64)
        out["sh"] = bf16_rne64(out["sh"]).astype(np.float64)
    return out


# ----------------------------------------------------------------------------
# split and merge (FP32 decisions, exact FP32 values)
# ----------------------------------------------------------------------------

def row_dims(codebook: int, sh_degree: int) -> tuple[int, int]:
    """(values moved, values stored) per row: SR 7 of 8, SH 3 (d+1)^2."""
    if codebook == 0:
        return SR_DIMS, SR_WIDTH
    b = 3 * (sh_degree + 1) ** 2
    return b, b


def _coefs(eps_split: float, eps_merge: float):
    es, em = np.float32(eps_split), np.float32(eps_merge)
    inv_s = np.float32(1.0) / (es * es)
    inv_m = np.float32(1.0) / (em * em)
    kc = np.float32(0.5) * (inv_s - inv_m)     # log q_sm(u) = -|u|^2 kc
    km = np.float32(0.5) * inv_m               # merge kernel: exp(-|c - c'|^2 km)
    return es, kc, km


def split_normals32(n: int, codebook: int, dims: int, step: int, seed: int) -> np.ndarray:
    """[n, dims] FP32 normals of every Gaussian's split proposal."""
    calls = (dims + 3) // 4
    z = np.empty((n, calls * 4), dtype=np.float32)
    for j in range(calls):
        z[:, 4 * j:4 * j + 4] = normals32(draws(np.arange(n), STREAM_SPLIT_U + codebook, j, step, seed))
    return z[:, :dims]


def split(rows, parent, g2x, k: int, k_cap: int, codebook: int, sh_degree: int, lam: float,
          eps_split: float, eps_merge: float, step: int, seed: int, bf16: bool = False) -> dict:
    """One split transition of one codebook (Sec. 4.4, Appendix A.1).

    Every Gaussian i proposes a new row c'' = c + u for its row c = g2x[i],
    u = eps_split z.  It is eligible if row c has at least two members and i
    is not the first of them (a row keeps one member).  Accepted iff
    v < min(1, exp(-lambda + |u|^2 kc)), i.e. min(1, e^-lambda / q_sm(u)).
    Accepted Gaussians get rows k, k + 1, ... in Gaussian order while rows
    last (k_cap); the new row's parent is c.  Returns rows, parent, g2x, k
    and the per-Gaussian flags."""
    dims, width = row_dims(codebook, sh_degree)
    rows = np.array(rows, dtype=np.float32).reshape(-1, width)
    assert rows.shape[0] >= k_cap
    parent = np.array(parent, dtype=np.int32).copy()
    g2x = np.array(g2x, dtype=np.int64).copy()
    n = g2x.size
    es, kc, _ = _coefs(eps_split, eps_merge)
    members = np.bincount(g2x, minlength=k)
    first = np.full(k, n, dtype=np.int64)
    np.minimum.at(first, g2x, np.arange(n))
    eligible = (members[g2x] >= 2) & (np.arange(n) != first[g2x])
    z = split_normals32(n, codebook, dims, step, seed)
    u = (es * z).astype(np.float32)
    n2 = np.zeros(n, dtype=np.float32)
    for d in range(dims):
        n2 = (n2 + u[:, d] * u[:, d]).astype(np.float32)
    la = (n2 * kc - np.float32(lam)).astype(np.float32)
    v = uniform32(draws(np.arange(n), STREAM_SPLIT_V + codebook, 0, step, seed)[:, 0])
    accept = eligible & (v < exp32(la))
    rank = np.cumsum(accept) - accept
    kept = accept & (k + rank < k_cap)
    idx = np.nonzero(kept)[0]
    new = k + rank[idx]
    c = g2x[idx]
    newrows = rows[c].copy()
    newrows[:, :dims] = (rows[c, :dims] + u[idx]).astype(np.float32)
    if bf16:
        newrows = bf16_rne(newrows).reshape(newrows.shape)
    rows[new] = newrows
    parent[new] = c
    g2x[idx] = new
    return {"rows": rows, "parent": parent, "g2x": g2x, "k": int(k + idx.size), "accepted": kept,
            "proposed_accept": accept, "eligible": eligible, "la": la, "v": v}


def merge(rows, parent, g2x, k: int, codebook: int, sh_degree: int, lam: float, eps_split: float,
          eps_merge: float, step: int, seed: int) -> dict:
    """One merge transition of one codebook (Sec. 4.4, Appendix A.1).

    Every row r < k with a parent p = parent[r] (the row it was split from)
    proposes to merge into p with probability exp(-|c_r - c_p|^2 km) (the
    unnormalised N(c - c' | 0, eps_merge^2 I)) and accepts with
    min(1, exp(lambda - |c_r - c_p|^2 kc)) = min(1, e^lambda q_sm(c - c')).
    A row merges only if its parent does not merge in the same step.  Its
    members move to the parent, the row is removed, surviving rows are
    compacted in order, and indices and parents are renumbered."""
    dims, width = row_dims(codebook, sh_degree)
    rows = np.array(rows, dtype=np.float32).reshape(-1, width)
    parent = np.array(parent, dtype=np.int64)
    g2x = np.array(g2x, dtype=np.int64)
    _, kc, km = _coefs(eps_split, eps_merge)
    r = np.arange(k)
    p = parent[:k]
    has = (p >= 0) & (p < k)
    pc = np.where(has, p, 0)
    d2 = np.zeros(k, dtype=np.float32)
    for d in range(dims):
        diff = (rows[:k, d] - rows[pc, d]).astype(np.float32)
        d2 = (d2 + diff * diff).astype(np.float32)
    rho = exp32(-(d2 * km).astype(np.float32))
    la = (np.float32(lam) - d2 * kc).astype(np.float32)
    bits = draws(r, STREAM_MERGE + codebook, 0, step, seed)
    v1, v2 = uniform32(bits[:, 0]), uniform32(bits[:, 1])
    tent = has & (v1 < rho) & (v2 < exp32(la))
    final = tent & ~tent[pc]
    target = np.where(final, pc, r)
    alive = ~final
    newidx = np.cumsum(alive) - alive
    k_new = int(alive.sum())
    out_rows = rows.copy()
    out_rows[newidx[alive]] = rows[:k][alive]
    out_parent = np.full(parent.shape, -1, dtype=np.int32)
    src = np.nonzero(alive)[0]
    par = parent[src]
    ok = (par >= 0) & (par < k)
    out_parent[newidx[src]] = np.where(ok, newidx[target[np.where(ok, par, 0)]], -1)
    out_g2x = newidx[target[g2x]]
    return {"rows": out_rows, "parent": out_parent, "g2x": out_g2x, "k": k_new, "merged": final,
            "proposed": tent, "d2": d2}


# ----------------------------------------------------------------------------
# growth (Sec. 5.1: +5 % Gaussians every 100 iterations by duplication)
# ----------------------------------------------------------------------------

STREAM_GROW = 24


def sigmoid32(logit) -> np.ndarray:
    """Opacity in the FP32 decision arithmetic: 1 / (1 + exp32(-l))."""
    l = np.asarray(logit, dtype=np.float32).ravel()
    return (np.float32(1.0) / (np.float32(1.0) + exp32(-l))).astype(np.float32)


def grow_weights(logit) -> np.ndarray:
    """Integer sampling weights floor(o 2^24) (exact in FP32, so both sides
    agree; uniform weights when every weight is 0)."""
    o = sigmoid32(logit)
    w = np.floor(o * np.float32(2.0 ** 24)).astype(np.int64)
    return w if w.sum() > 0 else np.ones_like(w)


def grow(pos, logit, g2sr, g2sh, m: int, step: int, seed: int) -> dict:
    """m new Gaussians, each a copy of an existing one drawn with
    probability proportional to its opacity: new Gaussian j takes the 64-bit
    draw x of counter (j, stream 24, step), u = x mod W (W = sum of the
    weights) and copies the Gaussian whose weight interval holds u.  The
    copies are appended after the n existing Gaussians."""
    n = len(logit)
    w = grow_weights(logit)
    incl = np.cumsum(w)
    total = int(incl[-1])
    d = draws(np.arange(m), STREAM_GROW, 0, step, seed).astype(np.uint64)
    x = (d[:, 1] << np.uint64(32)) | d[:, 0]
    u = (x % np.uint64(total)).astype(np.int64)
    src = np.searchsorted(incl, u, side="right")
    return {"src": src.astype(np.int64),
            "pos": np.concatenate([np.asarray(pos, np.float32).reshape(n, 3), np.asarray(pos, np.float32).reshape(n, 3)[src]]),
            "logit": np.concatenate([np.asarray(logit, np.float32), np.asarray(logit, np.float32)[src]]),
            "g2sr": np.concatenate([np.asarray(g2sr), np.asarray(g2sr)[src]]),
            "g2sh": np.concatenate([np.asarray(g2sh), np.asarray(g2sh)[src]])}
