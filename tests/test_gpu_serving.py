"""Serving (continuous batching) through the C ABI.

A served request runs the code ADMM to a residual tolerance; its slot and its
dictionary version are the only state it reads, so its result is the same
alone and among other requests in flight.  With learning on, completed
requests are folded in completion order and DictOCSC runs after every
update_every completions.
"""
import numpy as np
import pytest

import oracle
from tests.close import assert_close
from workloads import make_image, raw_filters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _learner(pkg, K=16, M=8, sizes=(64, 128), max_batch=8, **kw):
    raw = raw_filters(K, M, 31)
    lr = pkg.OCSC(K, M, 0.5, 1.0, fft_sizes=list(sizes), pad=M - 1, Jz=50, Jd=6, max_batch=max_batch, **kw)
    lr.set_dict(raw, normalize=True)
    return lr, raw


def _serve_all(srv, reqs, max_steps=400):
    """Submit (id, image) pairs and step until all complete; returns id -> result."""
    for rid, im in reqs:
        srv.submit(rid, im)
    out = {}
    for _ in range(max_steps):
        active, queued = srv.step()
        for d in srv.poll():
            out[d["id"]] = d
        if active == 0 and queued == 0:
            break
    return out


def test_result_same_alone_and_in_mix():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lr, _ = _learner(pkg)
    target = torch.from_numpy(make_image(50, 50, 1)).cuda()
    others = [torch.from_numpy(make_image(s, s, 10 + i)).cuda() for i, s in enumerate([100, 50, 110, 40, 90])]
    srv = pkg.Server(lr, learn=0, tol=1e-4, check_every=5, max_iters=300)
    alone = _serve_all(srv, [(7, target)])[7]
    srv.close()
    srv = pkg.Server(lr, learn=0, tol=1e-4, check_every=5, max_iters=300)
    mix = _serve_all(srv, [(1, others[0]), (2, others[1]), (7, target)] + [(3 + i, o) for i, o in enumerate(others[2:])])
    srv.close()
    assert len(mix) == 6
    assert mix[7]["iters"] == alone["iters"]
    assert torch.equal(mix[7]["code"], alone["code"])
    lr.close()


def test_result_same_alone_and_in_mix_while_learning():
    """learn = 1: dictionary updates run on the context's stream while other
    requests are in flight.  Every served request, recoded alone by a fresh
    server (learning off) against the dictionary version it reports, gives the
    same iterations and the same code bit for bit: the two-version fence keeps
    a request on the dictionary current at its admission."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lr, raw = _learner(pkg, K=12, M=5, sizes=(64, 128), max_batch=4)
    sides = [50, 100, 40, 90, 55, 110, 45, 60, 100, 50, 57, 95]
    imgs = [torch.from_numpy(make_image(s, s, 300 + i)).cuda() for i, s in enumerate(sides)]
    srv = pkg.Server(lr, learn=1, update_every=4, tol=1e-3, check_every=5, max_iters=150)
    versions = {0: lr.get_dict()}
    pending = list(range(len(imgs)))
    res = {}
    seen_updates = 0
    for i in pending[:6]:              # a first wave; its completions trigger an update
        srv.submit(i, imgs[i])
    pending = pending[6:]
    for _ in range(2000):
        updates = lr.counters()["dict_updates"]
        if updates > seen_updates and pending:   # later waves arrive while the
            seen_updates = updates               # earlier requests and the
            for i in pending[:3]:                # update are still in flight
                srv.submit(i, imgs[i])
            pending = pending[3:]
        active, queued = srv.step()
        for d in srv.poll():
            res[d["id"]] = d
        D = lr.get_dict()
        versions.setdefault(lr.version, D)
        if not pending and active == 0 and queued == 0:
            break
    srv.close()
    assert len(res) == len(imgs)
    used = sorted({d["dict_version"] for d in res.values()})
    assert len(used) >= 2, used        # the stream saw at least one update
    for i, d in res.items():
        alone_ctx, _ = _learner(pkg, K=12, M=5, sizes=(64, 128), max_batch=4)
        alone_ctx.set_dict(versions[d["dict_version"]], normalize=False)
        one = pkg.Server(alone_ctx, learn=0, tol=1e-3, check_every=5, max_iters=150)
        a = _serve_all(one, [(i, imgs[i])])[i]
        one.close()
        alone_ctx.close()
        assert a["iters"] == d["iters"], (i, a["iters"], d["iters"])
        assert torch.equal(a["code"], d["code"]), i
    lr.close()


@pytest.mark.parametrize("sizes,sides", [((64, 128), (50, 100, 57)), ((96, 144), (80, 130, 85))])
def test_served_codes_match_oracle_at_reported_iterations(sizes, sides):
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lr, raw = _learner(pkg, sizes=sizes)
    imgs = [make_image(s, s, 40 + i) for i, s in enumerate(sides)]
    srv = pkg.Server(lr, learn=0, tol=1e-4, check_every=5, max_iters=200)
    res = _serve_all(srv, [(i, torch.from_numpy(im).cuda()) for i, im in enumerate(imgs)])
    srv.close()
    D = oracle.normalize_filters(np.asarray(raw, np.float64))
    for i, im in enumerate(imgs):
        d = res[i]
        assert d["iters"] % 5 == 0 and 5 <= d["iters"] <= 200
        assert (d["primal"] <= 1e-4 and d["dual"] <= 1e-4) or d["iters"] == 200
        N = sizes[0] if max(im.shape) + 7 <= sizes[0] else sizes[1]
        o = oracle.code_admm(oracle.pad_to(np.asarray(im, np.float64), N, N),
                             oracle.filters_spectrum(D, N, N), 0.5, 1.0, d["iters"])
        assert_close(d["code"].cpu().numpy(), o.U, f"served request {i} ({d['iters']} iterations)")
    lr.close()


def test_learning_through_the_server_matches_oracle():
    """update_every = 4: the four completed requests are folded in completion
    order and DictOCSC runs once; compare with the oracle doing the same."""
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lr, raw = _learner(pkg, K=12, M=5, sizes=(64,), max_batch=4)
    imgs = [make_image(s, s, 70 + i) for i, s in enumerate([50, 57, 45, 52])]
    srv = pkg.Server(lr, learn=1, update_every=4, tol=1e-4, check_every=5, max_iters=100)
    res = _serve_all(srv, [(i, torch.from_numpy(im).cuda()) for i, im in enumerate(imgs)])
    srv.close()
    D = lr.get_dict()
    assert lr.version == 1
    order = list(res.values())          # completion order
    st = oracle.init_state(np.asarray(raw, np.float64), 64, 64, 0.5, 1.0)
    results = [oracle.code(st, imgs[d["id"]], d["iters"]) for d in order]
    oracle.update_dict(st, results, 6)
    assert_close(D, st.V, "dictionary learned through the server")
    lr.close()


def test_memory_budget_limits_requests_in_flight():
    _need_gpu()
    import paper_1706_06972_gb300 as pkg

    lr, _ = _learner(pkg, sizes=(64,))
    # one 64x64 request with K = 16 needs about 1.4 MB of working set
    srv = pkg.Server(lr, learn=0, mem_budget=2 << 20, tol=1e-3, check_every=5, max_iters=50)
    for i in range(4):
        srv.submit(i, torch.from_numpy(make_image(50, 50, 90 + i)).cuda())
    done, peak = 0, 0
    for _ in range(100):
        active, queued = srv.step()
        peak = max(peak, active)
        done += len(srv.poll())
        if active == 0 and queued == 0:
            break
    srv.close()
    assert done == 4 and peak == 1
    lr.close()
