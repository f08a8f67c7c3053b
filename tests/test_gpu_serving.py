"""Serving runtime: continuous batching of TSMM requests against device-resident
packed B matrices.  Every result must be the same, bit for bit, whether the
request ran alone or in the mix (its plan depends only on its shape), and
within the oracle's bound; admission must respect the memory budget; batches
must overlap on the device."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti
from gpu_util import to_device

pytestmark = pytest.mark.gpu

B_SPECS = [(64, 1), (200, 16), (777, 64), (1500, 8), (4000, 33), (100, 3)]


def make_bs(dtype=np.float32):
    out = []
    for i, (k, n) in enumerate(B_SPECS):
        B = ti.matrix_np(k, n, 500 + i, "uniform", dtype)
        out.append((k, n, B, tsmm.pack_b(to_device(B))))
    return out


def make_requests(bs, count, seed, dtype=np.float32):
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(count):
        b = int(rng.integers(len(bs)))
        k, n, B, pb = bs[b]
        m = int(np.exp(rng.uniform(np.log(100), np.log(8000))))
        A = ti.matrix_np(m, k, 1000 + rid, "uniform", dtype)
        C0 = ti.matrix_np(m, n, 2000 + rid, "uniform", dtype)
        reqs.append(dict(id=rid, b=b, m=m, A=A, C0=C0, alpha=1.5, beta=0.5 if rid % 3 else 0.0))
    return reqs


def run(server, bs, reqs, spread_s=0.0, seed=0):
    rng = np.random.default_rng(seed)
    t0 = tsmm.tsmm_server_clock() + 0.002
    devs, batch = {}, []
    for q in reqs:
        k, n, B, pb = bs[q["b"]]
        dA, dC = to_device(q["A"]), to_device(q["C0"])
        devs[q["id"]] = (dA, dC)
        batch.append((q["id"], pb, q["m"], q["alpha"], dA, q["beta"], dC,
                      t0 + (rng.uniform(0, spread_s) if spread_s else 0.0)))
    # the server's streams are not ordered after torch's: inputs must be in place
    torch.cuda.synchronize()
    server.submit(batch)
    server.drain(120.0)
    comps = {c["id"]: c for c in server.poll()}
    assert len(comps) == len(reqs) and all(c["status"] == 0 for c in comps.values())
    return {rid: d[1].cpu().numpy() for rid, d in devs.items()}, comps


def test_serving_same_alone_and_in_mix():
    bs = make_bs()
    reqs = make_requests(bs, 40, seed=1)
    # alone: one request at a time through a server
    alone = {}
    srv = tsmm.Server(budget_bytes=8 << 30, num_streams=4, max_batch=16)
    for q in reqs:
        res, _ = run(srv, bs, [q])
        alone[q["id"]] = res[q["id"]]
    srv.close()
    # in the mix: all of them, arriving over 20 ms, overlapping on the device
    srv = tsmm.Server(budget_bytes=8 << 30, num_streams=4, max_batch=16)
    mix, comps = run(srv, bs, reqs, spread_s=0.02, seed=2)
    srv.close()
    for q in reqs:
        k, n, B, pb = bs[q["b"]]
        Cref, E = oracle.tsmm(q["alpha"], q["A"], B, q["beta"], q["C0"] if q["beta"] else None)
        if not np.array_equal(mix[q["id"]], alone[q["id"]]):
            where = np.argwhere(mix[q["id"]] != alone[q["id"]])
            verdict = {tag: oracle.check(r, Cref, E, np.float32)[2] for tag, r in
                       (("alone", alone[q["id"]]), ("mix", mix[q["id"]]))}
            raise AssertionError(f"request {q['id']} (m={q['m']}, k={k}, n={n}, beta={q['beta']}) differs "
                                 f"in {len(where)} entries, first {where[:4].tolist()}; entries outside "
                                 f"the oracle's bound: {verdict}")
        ok, ratio, nbad = oracle.check(mix[q["id"]], Cref, E, np.float32)
        assert ok, f"request {q['id']}: {nbad} entries outside the bound"
    for c in comps.values():
        assert c["arrival_s"] <= c["admit_s"] <= c["launch_s"] <= c["complete_s"]


def test_serving_fp64_same_alone_and_in_mix():
    """An FP64 server: every request equal bit for bit alone and in the mix, and
    within the oracle's componentwise bound (Dot2-accurate reference)."""
    bs = make_bs(np.float64)
    reqs = make_requests(bs, 24, seed=7, dtype=np.float64)
    alone = {}
    srv = tsmm.Server(budget_bytes=8 << 30, dtype=torch.float64, num_streams=4, max_batch=16)
    for q in reqs:
        res, _ = run(srv, bs, [q])
        alone[q["id"]] = res[q["id"]]
    srv.close()
    srv = tsmm.Server(budget_bytes=8 << 30, dtype=torch.float64, num_streams=4, max_batch=16)
    mix, _ = run(srv, bs, reqs, spread_s=0.01, seed=8)
    srv.close()
    for q in reqs:
        assert np.array_equal(mix[q["id"]], alone[q["id"]]), f"request {q['id']} differs"
        k, n, B, pb = bs[q["b"]]
        Cref, E = oracle.tsmm(q["alpha"], q["A"], B, q["beta"], q["C0"] if q["beta"] else None)
        ok, ratio, nbad = oracle.check(mix[q["id"]], Cref, E, np.float64)
        assert ok, f"request {q['id']}: {nbad} entries outside the bound"


def test_serving_mix_repeats_bitwise_under_concurrency():
    """Eight mixes of the same 40 requests, each with its own arrival order,
    against one direct tsmm_execute per request: every result identical bit
    for bit.  Grouped launches of several kernel classes then run side by side
    on the server's streams, which is what exposed a consumer's shared-memory
    reads of a ring stage racing the copy that refills it (the release fence
    before each empty-barrier arrival); without that fence about one mix in
    four had one k term of one warp wrong."""
    bs = make_bs()
    reqs = make_requests(bs, 40, seed=1)
    direct = {}
    for q in reqs:
        k, n, B, pb = bs[q["b"]]
        dA, dC = to_device(q["A"]), to_device(q["C0"])
        pl = tsmm.plan(q["m"], n, k, torch.float32)
        tsmm.execute(pl, q["alpha"], dA, pb, q["beta"], dC)
        pl.check()
        direct[q["id"]] = dC.cpu().numpy()
    for trial in range(8):
        srv = tsmm.Server(budget_bytes=8 << 30, num_streams=4, max_batch=16)
        mix, _ = run(srv, bs, reqs, spread_s=0.02, seed=100 + trial)
        srv.close()
        for q in reqs:
            i = q["id"]
            if not np.array_equal(mix[i], direct[i]):
                rows = np.unique(np.argwhere(mix[i] != direct[i])[:, 0])
                raise AssertionError(f"mix {trial}: request {i} differs from its direct launch in rows "
                                     f"{rows[0]}..{rows[-1]} ({len(rows)} rows)")


def test_serving_admission_respects_budget_and_batches_overlap():
    bs = make_bs()
    reqs = make_requests(bs, 60, seed=3)
    es = 4
    sizes = {q["id"]: es * q["m"] * (bs[q["b"]][0] + bs[q["b"]][1]) for q in reqs}
    budget = 3 * max(sizes.values())
    srv = tsmm.Server(budget_bytes=budget, num_streams=4, max_batch=8)
    _, comps = run(srv, bs, reqs, spread_s=0.0, seed=4)
    srv.close()
    # at every admission, the requests admitted and not yet completed fit the budget
    ev = sorted(comps.values(), key=lambda c: c["admit_s"])
    for c in ev:
        live = sum(sizes[d["id"]] for d in ev if d["admit_s"] <= c["admit_s"] < d["complete_s"])
        assert live <= budget
    # with a roomy budget, admitted work overlaps on the device (several batches in flight)
    srv = tsmm.Server(budget_bytes=16 << 30, num_streams=4, max_batch=4)
    _, comps = run(srv, bs, reqs, spread_s=0.0, seed=5)
    srv.close()
    spans = sorted((c["launch_s"], c["complete_s"]) for c in comps.values())
    overlap = max(sum(1 for (a, b) in spans if a <= t < b) for (t, _) in spans)
    assert overlap >= 2


def test_serving_rejects_requests_larger_than_budget():
    bs = make_bs()
    k, n, B, pb = bs[2]
    A = to_device(ti.matrix_np(5000, k, 1, "uniform", np.float32))
    C = to_device(np.zeros((5000, n), np.float32, order="F"))
    srv = tsmm.Server(budget_bytes=1 << 20, num_streams=1, max_batch=1)
    with pytest.raises(tsmm.TsmmError) as e:
        srv.submit([(0, pb, 5000, 1.0, A, 0.0, C, 0.0)])
    assert e.value.status == 1
    # a future request is dropped cleanly when the server is closed before it arrives
    small = to_device(ti.matrix_np(10, k, 1, "uniform", np.float32))
    Cs = to_device(np.zeros((10, n), np.float32, order="F"))
    srv.submit([(1, pb, 10, 1.0, small, 0.0, Cs, tsmm.tsmm_server_clock() + 3600.0)])
    srv.close()


def test_serving_small_requests_finish_before_a_large_one_of_their_batch():
    """A batch goes out cheapest request first in sub-batches with their own
    completion events: small requests launched with a large one complete
    before it, with correct results."""
    bs = make_bs()
    k_s, n_s, B_s, pb_s = bs[5]
    m_big, k_big, n_big = 131072, 4096, 64
    A_big = torch.empty((k_big, m_big), dtype=torch.float32, device="cuda")
    ti.fill_torch(A_big, 7, "uniform")
    A_big = A_big.t()
    B_big = torch.empty((n_big, k_big), dtype=torch.float32, device="cuda")
    ti.fill_torch(B_big, 8, "uniform")
    pb_big = tsmm.pack_b(B_big.t())
    C_big = torch.zeros((n_big, m_big), dtype=torch.float32, device="cuda").t()
    smalls = []
    for rid in range(1, 17):
        A = ti.matrix_np(1024, k_s, 3000 + rid, "uniform", np.float32)
        smalls.append((rid, A, to_device(A), to_device(np.zeros((1024, n_s), np.float32, order="F"))))
    torch.cuda.synchronize()  # inputs in place before the server's streams read them
    srv = tsmm.Server(budget_bytes=40 << 30, num_streams=1, max_batch=64)
    t0 = tsmm.tsmm_server_clock() + 0.005
    batch = [(0, pb_big, m_big, 1.0, A_big, 0.0, C_big, t0)]
    batch += [(rid, pb_s, 1024, 1.0, dA, 0.0, dC, t0) for (rid, A, dA, dC) in smalls]
    srv.submit(batch)
    srv.drain(120.0)
    comps = {c["id"]: c for c in srv.poll()}
    srv.close()
    assert len(comps) == 17 and all(c["status"] == 0 for c in comps.values())
    assert len({c["launch_s"] for c in comps.values()}) == 1, "expected one batch"
    assert max(comps[rid]["complete_s"] for rid in range(1, 17)) < comps[0]["complete_s"]
    for (rid, A, dA, dC) in smalls:
        Cref, E = oracle.tsmm(1.0, A, B_s, 0.0, None)
        ok, ratio, nbad = oracle.check(dC.cpu().numpy(), Cref, E, np.float32)
        assert ok, f"request {rid}: {nbad} entries outside the bound"


def _split_k_request(rid, m, n, k, seed):
    A = ti.matrix_np(m, k, seed, "uniform", np.float32)
    B = ti.matrix_np(k, n, seed + 1, "uniform", np.float32)
    C0 = ti.matrix_np(m, n, seed + 2, "uniform", np.float32)
    pb = tsmm.pack_b(to_device(B))
    return dict(id=rid, A=A, B=B, C0=C0, pb=pb, dA=to_device(A), dC=to_device(C0))


def _submit(server, reqs, alpha=1.5, beta=0.5):
    torch.cuda.synchronize()  # inputs in place before submission (the server's ordering contract)
    t0 = tsmm.tsmm_server_clock()
    server.submit([(q["id"], q["pb"], q["A"].shape[0], alpha, q["dA"], beta, q["dC"], t0) for q in reqs])
    server.drain(60.0)
    return {c["id"]: c for c in server.poll()}


def test_serving_timeout_clears_split_k_counters():
    """A launch unit whose kernels gave up (injected on the host: status word set,
    arrival counters left part-way, as a block that gave up before its ticket
    leaves them) completes with TSMM_ERR_TIMEOUT, and the next split-K request,
    which the arena hands the same counter slice, is still exact: the server
    cleared the counters before releasing them."""
    m, n, k = 300, 16, 20000
    assert tsmm.plan(m, n, k, torch.float32).info()["splits"] > 1  # split-K: counters in use
    srv = tsmm.Server(budget_bytes=1 << 30, num_streams=1, max_batch=1)
    try:
        first = _split_k_request(0, m, n, k, 700)
        srv.inject_timeout(1)
        comps = _submit(srv, [first])
        assert comps[0]["status"] == 7  # TSMM_ERR_TIMEOUT
        for rid in (1, 2):  # follow-ups reuse the cleared slice
            q = _split_k_request(rid, m, n, k, 700 + 10 * rid)
            comps = _submit(srv, [q])
            assert comps[rid]["status"] == 0
            Cref, E = oracle.tsmm(1.5, q["A"], q["B"], 0.5, q["C0"])
            ok, ratio, nbad = oracle.check(q["dC"].cpu().numpy(), Cref, E, np.float32)
            assert ok, f"follow-up {rid}: {nbad} entries outside the bound (max ratio {ratio:.3g})"
    finally:
        srv.close()


def test_serving_timeout_charged_to_its_own_unit():
    """Two requests launched as separate units on two lanes, the first with an
    injected timeout: only that one reports TSMM_ERR_TIMEOUT; the other completes
    OK and matches the oracle (each launch unit has its own status word)."""
    m, n, k = 300, 16, 20000
    srv = tsmm.Server(budget_bytes=1 << 30, num_streams=2, max_batch=1)
    try:
        qs = [_split_k_request(rid, m, n, k, 800 + 10 * rid) for rid in range(2)]
        srv.inject_timeout(1)
        comps = _submit(srv, qs)
        assert comps[0]["status"] == 7 and comps[1]["status"] == 0
        Cref, E = oracle.tsmm(1.5, qs[1]["A"], qs[1]["B"], 0.5, qs[1]["C0"])
        ok, ratio, nbad = oracle.check(qs[1]["dC"].cpu().numpy(), Cref, E, np.float32)
        assert ok, f"{nbad} entries outside the bound (max ratio {ratio:.3g})"
    finally:
        srv.close()
