"""collo_eval_noalloc (evaluation into caller-owned device buffers, scratch in
a fixed device array) against collo_eval.  Named to be collected last, so it
also runs after every other test has used the library in this process."""
import numpy as np
import pytest

from paper_2607_12201_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ["phi", "c", "grad", "jac_z", "jac_theta", "hess_zz", "hess_ztheta", "hess_thth",
          "hess_obj"]


@pytest.fixture(scope="module")
def collo():
    from paper_2607_12201_gb300 import build
    build.build()
    from paper_2607_12201_gb300 import collo
    return collo


def _point(prob, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 1.5, prob.n_x)
    lam = rng.standard_normal(prob.n_c)
    return x, lam


def _device_outputs(torch, prob):
    n, p, N = prob.n, prob.p, prob.N
    shapes = dict(phi=(1,), c=(prob.n_c,), grad=(prob.n_x,), jac_z=(N, 3, n, n),
                  jac_theta=(N, 3, n, p), hess_zz=(N, 3, n, n), hess_ztheta=(N, 3, n, p),
                  hess_thth=(p,), hess_obj=(N, n, 4, 4))
    # NaN fill: a field the call failed to write cannot match
    return {k: torch.full(s, float("nan"), dtype=torch.float64, device="cuda")
            for k, s in shapes.items()}


def _compare(host, dev):
    for k in FIELDS:
        a = np.asarray(host[k], dtype=np.float64).reshape(-1)
        b = dev[k].cpu().numpy().reshape(-1)
        assert a.shape == b.shape, k
        scale = max(1.0, float(np.max(np.abs(a)))) if a.size else 1.0
        err = float(np.max(np.abs(a - b))) / scale if a.size else 0.0
        assert err <= 1e-15, (k, err)


@pytest.mark.parametrize("make", [lambda: W.config1(), lambda: W.config2(),
                                  lambda: W.small_network(n=3, r=4, N=1, seed=7)],
                         ids=["cascade_N50", "config2_N400", "tiny_N1"])
def test_noalloc_eval_matches_collo_eval_twice(collo, make):
    torch = pytest.importorskip("torch")
    inst = make()
    with collo.Problem(inst) as prob:
        stream = torch.cuda.current_stream().cuda_stream
        outs = _device_outputs(torch, prob)
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        results = []
        # two calls in a row at different points (the second one must not see
        # anything the first left in the shared scratch), then the first point
        # again without multipliers
        for seed, with_lam, of in [(1, True, 0.7), (2, True, 1.0), (1, False, 1.3)]:
            x, lam = _point(prob, seed)
            xd = torch.tensor(x, device="cuda")
            ld = torch.tensor(lam, device="cuda") if with_lam else None
            prob.eval_noalloc(xd.data_ptr(), None if ld is None else ld.data_ptr(), ptrs,
                              obj_factor=of, stream=stream)
            torch.cuda.synchronize()
            dev = {k: v.clone() for k, v in outs.items()}
            host = prob.eval(x, lam if with_lam else None, obj_factor=of)
            host["phi"] = np.array([host["phi"]])
            _compare(host, dev)
            results.append(dev)
        # same point twice in a row must give identical bits
        x, lam = _point(prob, 2)
        xd = torch.tensor(x, device="cuda")
        ld = torch.tensor(lam, device="cuda")
        prob.eval_noalloc(xd.data_ptr(), ld.data_ptr(), ptrs, obj_factor=1.0, stream=stream)
        torch.cuda.synchronize()
        for k in FIELDS:
            assert torch.equal(outs[k], results[1][k]), k


def test_noalloc_eval_rejects_oversized_null_and_host_pointers(collo):
    torch = pytest.importorskip("torch")
    # N (4 + p) + 8 above 2^19 doubles of fixed scratch
    inst = W.random_network(1, 2, n_obs=1, M=5, T=2.0, N=120000, seed=9)
    with collo.Problem(inst) as prob:
        assert prob.N * (4 + prob.p) + 8 > (1 << 19)
        outs = _device_outputs(torch, prob)
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        xd = torch.zeros(prob.n_x, dtype=torch.float64, device="cuda")
        with pytest.raises(collo.ColloError) as e:
            prob.eval_noalloc(xd.data_ptr(), None, ptrs)
        assert e.value.status == collo.ERR_INVALID_ARG
        assert "scratch" in collo.last_error()
    inst = W.small_network(n=3, r=4, N=4, seed=3)
    with collo.Problem(inst) as prob:
        outs = _device_outputs(torch, prob)
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        ptrs["jac_z"] = 0
        xd = torch.zeros(prob.n_x, dtype=torch.float64, device="cuda")
        with pytest.raises(collo.ColloError) as e:
            prob.eval_noalloc(xd.data_ptr(), None, ptrs)
        assert e.value.status == collo.ERR_INVALID_ARG
        # host memory where device memory is required: refused before any launch
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        xh = np.zeros(prob.n_x)
        with pytest.raises(collo.ColloError) as e:
            prob.eval_noalloc(xh.ctypes.data, None, ptrs)
        assert e.value.status == collo.ERR_INVALID_ARG
        assert "not device memory" in collo.last_error()
        pinned = torch.zeros(prob.n_c, dtype=torch.float64).pin_memory()
        ptrs["c"] = pinned.data_ptr()
        with pytest.raises(collo.ColloError) as e:
            prob.eval_noalloc(xd.data_ptr(), None, ptrs)
        assert e.value.status == collo.ERR_INVALID_ARG
        # the problem is still usable afterwards
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        x, lam = _point(prob, 4)
        xd = torch.tensor(x, device="cuda")
        prob.eval_noalloc(xd.data_ptr(), None, ptrs)
        torch.cuda.synchronize()
        host = prob.eval(x, None)
        host["phi"] = np.array([host["phi"]])
        _compare(host, outs)


def test_noalloc_eval_allocates_nothing_and_keeps_the_current_device(collo):
    """After one call (which looks up the scratch array's address), further
    calls leave the device's free memory unchanged and the caller's current
    device as it was."""
    torch = pytest.importorskip("torch")
    inst = W.config2(N=100)
    with collo.Problem(inst) as prob:
        outs = _device_outputs(torch, prob)
        ptrs = {k: v.data_ptr() for k, v in outs.items()}
        x, lam = _point(prob, 3)
        xd = torch.tensor(x, device="cuda")
        ld = torch.tensor(lam, device="cuda")
        prob.eval_noalloc(xd.data_ptr(), ld.data_ptr(), ptrs)
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        dev = torch.cuda.current_device()
        for _ in range(5):
            prob.eval_noalloc(xd.data_ptr(), ld.data_ptr(), ptrs)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == before
        assert torch.cuda.current_device() == dev
