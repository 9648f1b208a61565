"""Serving: concurrent requests of uneven sizes and kernels give the same
results as each request alone; repeated sources reuse one cached plan and the
queued repeats of one source are served together by one batched sum;
admission respects the memory budget."""
import math

import numpy as np
import pytest

from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _specs():
    rng = np.random.Generator(np.random.PCG64(90))
    specs = []
    for i in range(14):
        kernel = ["gaussian", "laplacian", "negdist"][i % 3]
        d = [20, 64, 200][(i // 3) % 3]
        precision = ["f32", "bf16", "f16x3"][i % 3] if kernel != "laplacian" else "f16x3"
        N = int(rng.integers(500, 30000))
        M = int(rng.integers(100, 5000))
        P = [16, 64, 128][i % 3]
        specs.append((kernel, d, precision, N, M, P))
    return specs


def _inputs(dev, kernel, d, N, M, P, seed):
    g = torch.Generator(device=dev).manual_seed(seed)
    x = torch.randn(N, d, device=dev, generator=g)
    y = torch.randn(M, d, device=dev, generator=g) + 0.25
    w = torch.rand(N, device=dev, generator=g)
    xi = workloads.directions(P, d, seed=seed)
    param = math.sqrt(d) if kernel == "gaussian" else (1.0 / math.sqrt(d) if kernel == "laplacian" else 0.0)
    return x, y, w, xi, param


def test_alone_and_in_the_mix_agree():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Plan, Server
    reqs = []
    for i, (kernel, d, precision, N, M, P) in enumerate(_specs()):
        x, y, w, xi, param = _inputs(dev, kernel, d, N, M, P, 1000 + i)
        # the same sources queried three times with different targets: the repeats wait for
        # the first request's plan and are then served together from the cache
        ys = [y, y.flip(0).contiguous() * 0.9, (y[: max(1, M // 3)] - 0.1).contiguous()]
        alone = Plan(x, w, kernel, param, P=P, precision=precision, directions=xi, radius=8.0)
        reqs.append(dict(x=x, w=w, ys=ys, kernel=kernel, param=param, P=P, precision=precision, xi=xi,
                         refs=[alone.sum(t).cpu().numpy() for t in ys], wsum=float(w.sum())))
        alone.close()
    torch.cuda.synchronize()
    srv = Server(workers=4)
    ids = []
    xis = []
    for k, r in enumerate(reqs):
        xi = np.ascontiguousarray(r["xi"])
        xis.append(xi)
        desc = slk.make_desc(r["kernel"], r["param"], r["x"].shape[1], r["P"], r["precision"], radius=8.0)
        desc.directions = xi.ctypes.data
        r["outs"] = [torch.empty(t.shape[0], device=dev) for t in r["ys"]]
        for j, (t, o) in enumerate(zip(r["ys"], r["outs"])):
            ids.append((k, j, srv.submit(r["x"], r["w"], t, o, desc, source_key=k + 1)))
    cached, batched = 0, 0
    for k, j, rid in ids:
        res = srv.poll(rid, timeout_us=120_000_000)
        assert res is not None and res["status"] == 0, res
        cached += res["plan_cached"]
        batched += res["batch_requests"] > 1
        r = reqs[k]
        assert rel_inf(r["outs"][j], r["refs"][j], r["wsum"]) <= 1e-5, (k, j, r["kernel"], r["precision"])
    # every repeat waited for its plan and used it; the two repeats of a source queued behind
    # its build were served by one sum over their concatenated targets
    assert cached == 2 * len(reqs), cached
    assert batched >= len(reqs), batched
    srv.close()


def test_admission_under_a_small_budget_and_errors():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Server, SlkError
    kernel, d, N, M, P = "negdist", 32, 20000, 2000, 32
    x, y, w, xi, param = _inputs(dev, kernel, d, N, M, P, 7)
    desc = slk.make_desc(kernel, param, d, P, "f32")
    xi = np.ascontiguousarray(xi)
    desc.directions = xi.ctypes.data
    need = slk.request_bytes(desc, N, M)
    srv = Server(workers=4, memory_budget=int(need * 1.5))  # one request at a time fits
    outs = [torch.empty(M, device=dev) for _ in range(6)]
    ids = [srv.submit(x, w, y, o, desc) for o in outs]
    results = [srv.poll(i, timeout_us=120_000_000) for i in ids]
    assert all(r["status"] == 0 for r in results)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    # a request larger than the whole budget is refused at submission
    big = slk.make_desc(kernel, param, d, P, "f32")
    with pytest.raises(SlkError) as e:
        srv.submit(torch.zeros(200000, d, device=dev), torch.zeros(200000, device=dev), y, outs[0], big)
    assert e.value.status == 2
    with pytest.raises(SlkError) as e:
        srv.poll(123456789, timeout_us=0)
    assert e.value.status == 8
    srv.close()
