"""Serving with continuous batching: requests arrive while others run, are admitted as
slots and budget free up, share every launch with whatever else is running, and each
result is the same -- bitwise, with the same iteration count -- as the request solved
alone with lap_solve."""
import numpy as np
import pytest
import torch

from paper_2208_02427_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

K = 20  # SOR sweeps per server step


@pytest.fixture(scope="module")
def b():
    from paper_2208_02427_gb300 import binding
    binding.load()
    return binding


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def requests():
    out = []
    sizes = [(65, 65), (129, 33), (33, 129), (257, 257), (65, 129), (33, 33), (129, 129), (24, 17)]
    for k, (m, n) in enumerate(sizes * 2):
        method = ("mg_mixed", "mg", "sor")[k % 3]
        tol = (1e-10, 1e-8, 1e-6)[k % 3 if method != "sor" else 2]
        w = wl.w_opt_sor(m, n) if method == "sor" else 1.0
        out.append(dict(psi=wl.random_ring(m, n, seed=300 + k), method=method, tol=tol, w=w))
    return out


def alone(lap, b, r):
    t = b.to_field(r["psi"])
    g = lap.solve(t, method=r["method"], w=r["w"], tol=r["tol"], max_iter=200000,
                  check_every=K if r["method"] == "sor" else 1)
    return host(t), g


def test_results_in_the_mix_equal_results_alone(b):
    lap = b.Laplace()
    srv = b.Server(lap, hbm_budget=64 << 20, max_running=6, sor_sweeps=K)
    reqs = requests()
    fields, ids, results = {}, {}, {}
    pending = list(range(len(reqs)))
    step = 0
    max_running_seen = 0
    while pending or len(results) < len(reqs):
        # two new arrivals every step while others are mid-solve
        for _ in range(2):
            if pending:
                k = pending.pop(0)
                fields[k] = b.to_field(reqs[k]["psi"])
                ids[k] = srv.submit(fields[k], method=reqs[k]["method"], w=reqs[k]["w"],
                                    tol=reqs[k]["tol"], max_iter=200000)
        running, queued = srv.step()
        max_running_seen = max(max_running_seen, running)
        for k, rid in list(ids.items()):
            res = srv.poll(rid)
            if res is not None:
                results[k] = res
                del ids[k]
        step += 1
        assert step < 20000
    assert max_running_seen >= 3  # requests really overlapped
    for k, r in enumerate(reqs):
        want, g = alone(lap, b, r)
        got = results[k]
        assert got["status"] == g["status"] == "converged", (k, got, g)
        assert got["iters"] == g["iters"], (k, got, g)
        assert np.array_equal(host(fields[k]), want), k
    srv.close()
    lap.close()


def mixed_hierarchy_bytes(m, n, coarsest_min=5):
    """FP32 hierarchy of a mixed-precision request: u, q (and r except on the coarsest
    level) per level, rows padded to 32 floats, buffers 256-byte aligned."""
    total, levels = 0, []
    while True:
        levels.append((m, n))
        if (m - 1) % 2 or (n - 1) % 2 or (m - 1) // 2 + 1 < coarsest_min or (n - 1) // 2 + 1 < coarsest_min:
            break
        m, n = (m - 1) // 2 + 1, (n - 1) // 2 + 1
    for k, (m, n) in enumerate(levels):
        buf = -(-(n * (-(-m // 32) * 32) * 4) // 256) * 256
        total += buf * (2 if k == len(levels) - 1 else 3)
    return total


def test_admission_respects_the_budget(b):
    lap = b.Laplace()
    psi = wl.random_ring(257, 257, seed=1)
    one = mixed_hierarchy_bytes(257, 257)
    srv = b.Server(lap, hbm_budget=int(1.5 * one), max_running=8)
    fields = [b.to_field(psi) for _ in range(3)]
    ids = [srv.submit(f, method="mg_mixed", tol=1e-10) for f in fields]
    running, queued = srv.step()
    assert running == 1 and queued == 2  # one hierarchy fits the budget, the others wait
    done = {}
    while len(done) < 3:
        running, queued = srv.step()
        assert running <= 1
        for i in ids:
            if i not in done:
                r = srv.poll(i)
                if r is not None:
                    done[i] = r
    assert all(r["status"] == "converged" for r in done.values())
    outs = [host(f) for f in fields]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    srv.close()
    tiny = b.Server(lap, hbm_budget=1 << 16)
    with pytest.raises(b.LapError) as e:
        tiny.submit(b.to_field(psi), method="mg")
    assert e.value.code == -2
    tiny.close()
    lap.close()


def test_completion_list_gives_the_same_results_as_polling(b):
    """drain() reads the requests each step's convergence tests retired (a device-written
    list, one copy per step): every request comes out exactly once, in step order, with the
    result it has alone -- converged requests and ones stopped by their iteration cap."""
    lap = b.Laplace()
    srv = b.Server(lap, hbm_budget=64 << 20, max_running=5, sor_sweeps=K)
    reqs = requests()
    fields, ids = {}, {}
    order, results = [], {}
    pending = list(range(len(reqs)))
    capped = {3: 4, 2: 2 * K}  # max_iter: V-cycles (a mixed request), or sweeps (an SOR one)
    for step in range(20000):
        for _ in range(2):
            if pending:
                k = pending.pop(0)
                fields[k] = b.to_field(reqs[k]["psi"])
                ids[srv.submit(fields[k], method=reqs[k]["method"], w=reqs[k]["w"],
                               tol=reqs[k]["tol"], max_iter=capped.get(k, 200000))] = k
        srv.step()
        for rid, res in srv.drain(capacity=3):  # a small capacity: several calls per drain
            assert rid in ids
            order.append(rid)
            results[ids[rid]] = res
        if not pending and len(results) == len(reqs):
            break
    assert sorted(results) == list(range(len(reqs)))
    assert len(order) == len(set(order))
    for k, r in enumerate(reqs):
        t = b.to_field(r["psi"])
        g = lap.solve(t, method=r["method"], w=r["w"], tol=r["tol"], max_iter=capped.get(k, 200000),
                      check_every=K if r["method"] == "sor" else 1)
        assert results[k]["status"] == g["status"], (k, results[k], g)
        assert results[k]["iters"] == g["iters"], (k, results[k], g)
        assert np.array_equal(host(fields[k]), host(t)), k
    assert srv.drain() == []
    srv.close()
    lap.close()


def test_requests_at_the_edges_of_the_contract(b):
    """Each request against the same request solved alone with lap_solve (status, iterations
    and field, bit for bit): SOR caps that are not a multiple of the step's sweeps (the last
    step cut short, as lap_solve cuts its last check period), a cap of no iterations for every
    method (the initial residual, the field untouched), fields that already solve the problem
    (converged at once), dx != dy, and a NaN on the ring (DIVERGED at once). A method the server
    does not run and an unknown id are refused."""
    lap = b.Laplace()
    srv = b.Server(lap, hbm_budget=64 << 20, max_running=32, sor_sweeps=K)
    base = wl.random_ring(65, 33, seed=11)
    w = wl.w_opt_sor(65, 33)
    nan = wl.random_ring(33, 33, seed=15)
    nan[0, 5] = np.nan
    cases = [dict(psi=base, method="sor", w=w, tol=1e-12, max_iter=it) for it in (30, 7, K + 1)]
    for method in ("sor", "mg", "mg_mixed"):
        ww = w if method == "sor" else 1.0
        cases.append(dict(psi=base, method=method, w=ww, tol=1e-10, max_iter=0))
        cases.append(dict(psi=np.zeros((33, 65)), method=method, w=ww, tol=1e-10, max_iter=100))
        cases.append(dict(psi=nan, method=method, w=1.5 if method == "sor" else 1.0, tol=1e-10,
                          max_iter=100))
    cases += [dict(psi=wl.random_ring(65, 65, seed=12), method="mg", tol=1e-10, max_iter=50, dy=0.5),
              dict(psi=wl.random_ring(65, 65, seed=13), method="mg_mixed", tol=1e-10, max_iter=50, dx=0.5),
              dict(psi=wl.random_ring(65, 65, seed=14), method="sor", w=1.7, tol=1e-6, max_iter=2000,
                   dy=0.8)]
    fields, ids = [], []
    for c in cases:
        f = b.to_field(c["psi"])
        fields.append(f)
        ids.append(srv.submit(f, c.get("dx", 1.0), c.get("dy", 1.0), method=c["method"],
                              w=c.get("w", 1.0), tol=c["tol"], max_iter=c["max_iter"]))
    results = {}
    for _ in range(5000):
        srv.step()
        results.update(dict(srv.drain()))
        if len(results) == len(cases):
            break
    for k, (c, f, rid) in enumerate(zip(cases, fields, ids)):
        t = b.to_field(c["psi"])
        g = lap.solve(t, c.get("dx", 1.0), c.get("dy", 1.0), method=c["method"], w=c.get("w", 1.0),
                      tol=c["tol"], max_iter=c["max_iter"],
                      check_every=K if c["method"] == "sor" else 1)
        got = results[rid]
        assert (got["status"], got["iters"]) == (g["status"], g["iters"]), (k, c["method"], got, g)
        assert np.array_equal(host(f), host(t), equal_nan=True), k
    assert [results[i]["iters"] for i in ids[:3]] == [30, 7, K + 1]
    assert all(results[i]["status"] == "max_iter" for i in ids[:3])
    for j in range(3):
        zero_cap, solved, diverged = (results[ids[3 + 3 * j + d]] for d in range(3))
        assert (zero_cap["status"], zero_cap["iters"]) == ("max_iter", 0)
        assert zero_cap["r_final"] == zero_cap["r0"] > 0
        assert (solved["status"], solved["iters"]) == ("converged", 0)
        assert (diverged["status"], diverged["iters"]) == ("diverged", 0)
    with pytest.raises(b.LapError):
        srv.submit(b.to_field(base), method="adi", w=1.3)
    with pytest.raises(b.LapError):
        srv.poll(10 ** 12)
    srv.close()
    lap.close()
