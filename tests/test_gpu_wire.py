"""16-bit wire format on the GPU vs the CPU oracle (Sec. II.B, "Design of the
code on GF(65537)"): symbols as 16 bits, the positions of 65536 listed apart.

Expected values come from the oracle only: ``oracle.encode`` /
``oracle.encode_rows`` turned into wire form by ``oracle.wire``.  Columns
with escapes at known rows are planted in the source: s(x) = a + b x with
a = -1 - b r^j has the single root r^j of s(x) + 1, so e_j = 65536 there and
nowhere else in that column.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import small, wire

pytestmark = pytest.mark.gpu
P = 65537


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0907_1788_gb300 import build

    build.build()
    import paper_0907_1788_gb300 as pkg

    pkg.load()
    oracle.build()
    return pkg


def plant(src, n, col_rows, seed):
    """Column c becomes a + b x with its one escape at row j, for (c, j) in col_rows."""
    rng = np.random.default_rng(seed)
    r = small.root(n)
    for c, j in col_rows:
        while True:
            b = int(rng.integers(1, 65536))
            a = (-1 - b * pow(r, j, P)) % P
            if a <= 65535:
                break
        src[:, c] = 0
        src[0, c], src[1, c] = a, b
    return src


def _sorted(esc):
    e = np.asarray(esc, dtype=np.uint32).reshape(-1, 2)
    return e[np.lexsort((e[:, 1], e[:, 0]))]


def _planted_source(n, k, W, seed):
    src = synth.source(seed, k, W)
    rng = np.random.default_rng(seed + 1)
    cols = rng.choice(W, min(W, 6), replace=False)
    rows = [0, n - 1, n // 2, 1, int(rng.integers(0, n)), int(rng.integers(0, n))]
    return plant(src, n, list(zip(cols.tolist(), rows)), seed + 2), cols, rows


@pytest.mark.parametrize("n,k,W", [(64, 20, 17), (512, 256, 40), (8192, 4096, 64)])
def test_encode_wire_matches_oracle(pkg, n, k, W):
    src, _, _ = _planted_source(n, k, W, n + k)
    plan = pkg.Plan(n, k)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    want_sym, want_esc = wire.to_wire(oracle.encode(src, n))
    assert np.array_equal(pkg.to_host(sym), want_sym)
    assert np.array_equal(pkg.to_host(esc).reshape(-1, 2), want_esc)
    assert len(want_esc) >= 6


@pytest.mark.parametrize("n,k,W", [(16384, 12000, 8), (32768, 16384, 4), (65536, 32768, 6)])
def test_encode_wire_large(pkg, n, k, W):
    src, cols, rows = _planted_source(n, k, W, n + 7)
    plan = pkg.Plan(n, k)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    sym, esc = pkg.to_host(sym), pkg.to_host(esc).reshape(-1, 2)
    got = {tuple(e) for e in esc.tolist()}
    # every planted escape is listed, every listed escape is one (oracle rows)
    for c, j in zip(cols.tolist(), rows):
        assert (j, c) in got
    for j, c in got:
        assert oracle.encode_rows(np.ascontiguousarray(src[:, [c]]), n,
                                  np.array([j], np.uint32))[0, 0] == 65536
        assert sym[j, c] == 0
    samp = np.sort(np.random.default_rng(n).choice(n, 5, replace=False)).astype(np.uint32)
    want = oracle.encode_rows(src, n, samp)
    assert np.array_equal(sym[samp], (want & 0xFFFF).astype(np.uint16))


def test_encode_wire_every_schedule(pkg):
    for n, k, W, scheds in [(8192, 4096, 48, ("TMA", "TILE")),
                            (16384, 8192, 8, ("TILE", "SPLIT"))]:
        src, _, _ = _planted_source(n, k, W, 3 * n)
        plan = pkg.Plan(n, k)
        outs = []
        for s in scheds:
            plan.set_schedule(pkg.OP_ENCODE, getattr(pkg, "SCHED_" + s))
            sym, esc = plan.encode_wire(pkg.to_device(src))
            outs.append((pkg.to_host(sym), pkg.to_host(esc)))
        for sym, esc in outs[1:]:
            assert np.array_equal(sym, outs[0][0]) and np.array_equal(esc, outs[0][1])
        c = [0, 1, W // 2, W - 1]
        want = oracle.encode_rows(np.ascontiguousarray(src[:, c]), n,
                                  np.arange(0, n, 97, dtype=np.uint32))
        assert np.array_equal(outs[0][0][::97][:, c], (want & 0xFFFF).astype(np.uint16))


def test_escape_overflow_keeps_symbols(pkg):
    n, k, W = 512, 200, 64
    src = plant(synth.source(9, k, W), n, [(c, c % n) for c in range(40)], 10)
    plan = pkg.Plan(n, k)
    d_src = pkg.to_device(src)
    enc = torch.empty((n, W), dtype=torch.int16, device="cuda")
    esc = torch.zeros((5, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.fnt_rs_encode_wire(plan.handle, d_src, enc, esc, cnt,
                           plan.workspace(W, pkg.OP_ENCODE_WIRE))
    want_sym, want_esc = wire.to_wire(oracle.encode(src, n))
    assert int(cnt.item()) == len(want_esc) >= 40
    assert np.array_equal(pkg.to_host(enc), want_sym)
    listed = {tuple(e) for e in pkg.to_host(esc).reshape(-1, 2).tolist()}
    assert len(listed) == 5 and listed <= {tuple(e) for e in want_esc.tolist()}
    # the Plan helper re-runs with room for all of them
    _, esc_all = plan.encode_wire(d_src, cap=5)
    assert np.array_equal(pkg.to_host(esc_all).reshape(-1, 2), want_esc)


def test_punctured_wire(pkg):
    n, k, n_out, W = 1024, 512, 700, 24
    src = plant(synth.source(21, k, W), n, [(0, 5), (1, 699), (2, 700), (3, 1023)], 22)
    plan = pkg.Plan(n, k)
    plan.set_length(n_out)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    want_sym, want_esc = wire.to_wire(oracle.encode(src, n)[:n_out])
    assert sym.shape[0] == n_out
    assert np.array_equal(pkg.to_host(sym), want_sym)
    assert np.array_equal(pkg.to_host(esc).reshape(-1, 2), want_esc)
    got = {tuple(e) for e in want_esc.tolist()}
    assert (5, 0) in got and (699, 1) in got and (700, 2) not in got


@pytest.mark.parametrize("n,k,W", [(64, 20, 17), (512, 256, 40), (8192, 4096, 64),
                                   (65536, 32768, 3)])
def test_decode_wire_round_trip(pkg, n, k, W):
    seed = 11 * n + k
    src, cols, rows = _planted_source(n, k, W, seed)
    plan = pkg.Plan(n, k)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    sym, esc = pkg.to_host(sym), pkg.to_host(esc).reshape(-1, 2)
    pos = synth.received_positions(n, synth.erased_uniform(seed + 3, n, k))
    # make sure received packets carry escapes: swap planted rows into the first k
    planted = [j for j in rows if j not in set(pos[:k].tolist())][:2]
    for i, j in enumerate(planted):
        where = np.nonzero(pos == j)[0]
        if len(where):
            pos[[i, where[0]]] = pos[[where[0], i]]
        else:
            pos[i] = j
    resc = wire.select_rows(esc, pos)
    assert len(resc) >= 1
    out = plan.decode_wire(pkg.to_device(np.ascontiguousarray(sym[pos])), pos,
                           pkg.to_device(resc) if len(resc) else None)
    assert np.array_equal(pkg.to_host(out), src)
    assert plan.status() == 0


def test_decode_wire_matches_oracle_on_arbitrary_words(pkg):
    n, k, W = 1024, 400, 33  # odd W: the one-symbol widening path
    rng = np.random.default_rng(5)
    v = rng.integers(0, P, (k, W), dtype=np.uint32)
    v.reshape(-1)[rng.choice(v.size, 30, replace=False)] = 65536
    pos = rng.permutation(n)[:k].astype(np.uint32)
    sym, esc = wire.to_wire(v)
    plan = pkg.Plan(n, k)
    rev = esc[::-1].copy()  # any order
    got = pkg.to_host(plan.decode_wire(pkg.to_device(sym), pos, pkg.to_device(rev)))
    want, flag = oracle.decode(v, pos, n, k)
    assert np.array_equal(got, want)
    assert (plan.status() == pkg.E_RANGE) == bool(flag)


def test_decode_wire_rejects_bad_escapes(pkg):
    n, k, W = 256, 100, 16
    src = synth.source(31, k, W)
    plan = pkg.Plan(n, k)
    sym, _ = plan.encode_wire(pkg.to_device(src))
    pos = np.arange(k, dtype=np.uint32)
    rsym = sym[:k].contiguous()
    for bad in ([[k, 0]], [[0, W]]):  # outside the received rows / columns
        plan.decode_wire(rsym, pos, pkg.to_device(np.array(bad, np.uint32)))
        assert plan.status() == pkg.E_RANGE
    nz = np.argwhere(pkg.to_host(rsym) != 0)[0]  # a symbol that was not sent as 0
    plan.decode_wire(rsym, pos, pkg.to_device(np.array([nz], np.uint32)))
    assert plan.status() == pkg.E_RANGE
    # escapes of received rows beyond k are not used and not an error
    sym, esc = plan.encode_wire(pkg.to_device(src))
    pos2 = np.arange(k + 1, dtype=np.uint32)
    resc = wire.select_rows(pkg.to_host(esc), pos2)
    resc = np.concatenate([resc, np.array([[k, 3]], np.uint32)])
    out = plan.decode_wire(sym[:k + 1].contiguous(), pos2, pkg.to_device(resc))
    assert plan.status() == 0 and np.array_equal(pkg.to_host(out), src)


def test_wire_host_round_trip(pkg):
    n, k, W = 8192, 4096, 256
    src, cols, rows = _planted_source(n, k, W, 77)
    plan = pkg.Plan(n, k)
    h_src = torch.from_numpy(src.view(np.int16)).pin_memory()
    h_enc = torch.empty((n, W), dtype=torch.int16).pin_memory()
    cap = pkg.fnt_rs_wire_escape_cap(plan.handle, W)
    h_esc = np.zeros((cap, 2), dtype=np.uint32)
    ws = plan.workspace(W, pkg.OP_ENCODE_WIRE_HOST)
    m = pkg.fnt_rs_encode_wire_host(plan.handle, h_src, h_enc, h_esc, ws)
    c = sorted({int(x) for x in cols[:3]} | {W - 1})
    want_sym, want_esc = wire.to_wire(oracle.encode(np.ascontiguousarray(src[:, c]), n))
    sym = h_enc.numpy().view(np.uint16)
    assert np.array_equal(sym[:, c], want_sym)
    esc = h_esc[:m]
    assert np.array_equal(esc, _sorted(esc))  # sorted by row, then column
    mine = np.array([(r_, c.index(cc)) for r_, cc in esc.tolist() if cc in c], np.uint32)
    assert np.array_equal(_sorted(mine), want_esc)
    # too small an array: E_ARG, the count still reported
    if m:
        with pytest.raises(pkg.FntRsError):
            pkg.fnt_rs_encode_wire_host(plan.handle, h_src, h_enc, h_esc[:m - 1], ws)
    pos = synth.received_positions(n, synth.erased_uniform(78, n, k))
    pos = np.concatenate([np.array(rows[:2], np.uint32),
                          pos[~np.isin(pos, rows[:2])]]).astype(np.uint32)
    h_recv = torch.from_numpy(np.ascontiguousarray(sym[pos]).view(np.int16)).pin_memory()
    h_out = torch.empty((k, W), dtype=torch.int16).pin_memory()
    pkg.fnt_rs_decode_wire_host(plan.handle, h_recv, pos, wire.select_rows(esc, pos), h_out,
                                plan.workspace(W, pkg.OP_DECODE_WIRE_HOST))
    assert np.array_equal(h_out.numpy().view(np.uint16), src)
    assert plan.status() == 0


@pytest.mark.parametrize("W", [2048, 2500])
def test_host_calls_in_chunks(pkg, W):
    """The host-buffer calls cut W into column chunks (copies overlap the
    kernels); every chunk boundary and the ragged last chunk must agree with
    the oracle, in both formats."""
    n, k = 1024, 512
    src, cols, rows = _planted_source(n, k, W, W)
    plan = pkg.Plan(n, k)
    h_src = torch.from_numpy(src.view(np.int16)).pin_memory()
    c = sorted({0, 511, 512, 639, 640, 1023, 1024, 1279, 1280, 1535, 1536, 1919, 1920, W - 1}
               | {int(x) for x in cols})
    want = oracle.encode(np.ascontiguousarray(src[:, c]), n)
    # 32-bit symbols
    h_enc = torch.empty((n, W), dtype=torch.int32).pin_memory()
    pkg.fnt_rs_encode_host(plan.handle, h_src, h_enc, plan.workspace(W, pkg.OP_ENCODE_HOST))
    enc = h_enc.numpy().view(np.uint32)
    assert np.array_equal(enc[:, c], want)
    pos = synth.received_positions(n, synth.erased_uniform(W + 1, n, k))
    h_out = torch.empty((k, W), dtype=torch.int16).pin_memory()
    h_recv = torch.from_numpy(np.ascontiguousarray(enc[pos]).view(np.int32)).pin_memory()
    pkg.fnt_rs_decode_host(plan.handle, h_recv, pos, h_out,
                           plan.workspace(W, pkg.OP_DECODE_HOST))
    assert np.array_equal(h_out.numpy().view(np.uint16), src)
    # 16-bit wire symbols
    h_enc16 = torch.empty((n, W), dtype=torch.int16).pin_memory()
    h_esc = np.zeros((pkg.fnt_rs_wire_escape_cap(plan.handle, W), 2), dtype=np.uint32)
    m = pkg.fnt_rs_encode_wire_host(plan.handle, h_src, h_enc16, h_esc,
                                    plan.workspace(W, pkg.OP_ENCODE_WIRE_HOST))
    sym = h_enc16.numpy().view(np.uint16)
    want_sym, want_esc = wire.to_wire(want)
    assert np.array_equal(sym[:, c], want_sym)
    mine = np.array([(r_, c.index(cc)) for r_, cc in h_esc[:m].tolist() if cc in c],
                    np.uint32).reshape(-1, 2)
    assert np.array_equal(_sorted(mine), want_esc)
    assert np.array_equal(wire.from_wire(sym, h_esc[:m]), enc)  # all columns: same symbols
    pos = np.concatenate([np.array(rows[:2], np.uint32),
                          pos[~np.isin(pos, rows[:2])]]).astype(np.uint32)
    h_recv16 = torch.from_numpy(np.ascontiguousarray(sym[pos]).view(np.int16)).pin_memory()
    h_out.zero_()
    pkg.fnt_rs_decode_wire_host(plan.handle, h_recv16, pos, wire.select_rows(h_esc[:m], pos),
                                h_out, plan.workspace(W, pkg.OP_DECODE_WIRE_HOST))
    assert np.array_equal(h_out.numpy().view(np.uint16), src)
    assert plan.status() == 0


@pytest.mark.parametrize("n,k,W", [(512, 200, 24), (16384, 5000, 4)])
def test_wire_with_a_custom_root(pkg, n, k, W):
    """Another root of order n defines another MDS code (rows permuted by the
    index map); the wire output must follow it, escapes at the permuted rows."""
    r = oracle.root(n)
    root = pow(r, 7, P)
    src = synth.source(n + 3, k, W)
    plan = pkg.Plan(n, k, root=root)
    sym, esc = plan.encode_wire(pkg.to_device(src))
    sym, esc = pkg.to_host(sym), pkg.to_host(esc).reshape(-1, 2)
    rows = np.sort(np.random.default_rng(n).choice(n, 40, replace=False)).astype(np.uint32)
    want = oracle.encode_rows(src, n, rows, root_=root)
    assert np.array_equal(sym[rows], (want & 0xFFFF).astype(np.uint16))
    for j, c in esc.tolist():
        assert oracle.encode_rows(np.ascontiguousarray(src[:, [c]]), n, np.array([j], np.uint32),
                                  root_=root)[0, 0] == 65536
    pos = synth.received_positions(n, synth.erased_uniform(n + 4, n, k))
    resc = wire.select_rows(esc, pos)
    out = plan.decode_wire(pkg.to_device(np.ascontiguousarray(sym[pos])), pos,
                           pkg.to_device(resc) if len(resc) else None)
    assert np.array_equal(pkg.to_host(out), src)
    assert plan.status() == 0
