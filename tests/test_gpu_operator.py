"""GPU parity of the Wilson operator kernels (A and A^+, FP64 and FP32 two-row links)
against the CPU oracle, element by element, on lattices that span several
thread blocks, L = 2 wrap-around, odd/asymmetric extents and the largest workload."""
import numpy as np
import pytest

from tests.gpu_util import random_field, rel, small_problem, true_resid, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 6, 8), (6, 3, 5, 7), (8, 8, 8, 8)])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_fp64_matches_oracle(dims, dagger):
    from paper_0911_2285_gb300 import Solver
    links, op = small_problem(dims)
    v = np.stack([random_field(op.n, 1), random_field(op.n, 2), random_field(op.n, 3)])
    with Solver(links, dims, 0.12, nev=4, m=12, precision="mixed", k_max=2) as s:
        out = s.apply(v, dagger=dagger)
        for i in range(3):
            ref = op.apply_dag(v[i]) if dagger else op.apply(v[i])
            assert np.abs(out[i] - ref).max() <= 1e-14 * np.abs(ref).max()
            out32 = s.apply(v[i], dagger=dagger, precision="mixed")[0]
            assert rel(out32, ref) <= 2e-6


def test_apply_kappa_zero_is_identity():
    from paper_0911_2285_gb300 import Solver
    dims = (4, 2, 2, 2)
    links, op = small_problem(dims)
    v = random_field(op.n, 5)
    with Solver(links, dims, 0.0, nev=4, m=12, precision="fp64", k_max=1) as s:
        assert np.array_equal(s.apply(v)[0], v)


def test_apply_device_pointers_torch():
    torch = pytest.importorskip("torch")
    from paper_0911_2285_gb300 import Solver
    dims = (4, 4, 4, 8)
    links, op = small_problem(dims)
    v = random_field(op.n, 9)
    with Solver(links, dims, 0.12, nev=4, m=12, precision="fp64", k_max=1) as s:
        tv = torch.from_numpy(v).to("cuda:0")
        out = s.apply(tv)
        assert out.is_cuda
        torch.cuda.synchronize()
        ref = op.apply(v)
        assert np.abs(out.cpu().numpy()[0] - ref).max() <= 1e-14 * np.abs(ref).max()


def test_buffer_kind_must_match_on_device():
    """The C ABI refuses a host buffer declared as device memory (the kernels would
    read it) and a device buffer declared as host memory, before any copy or launch;
    the context stays usable."""
    torch = pytest.importorskip("torch")
    import ctypes as C
    from paper_0911_2285_gb300 import Solver
    from paper_0911_2285_gb300.lqcd import ERR_ARG, lib
    dims = (4, 4, 4, 4)
    links, op = small_problem(dims)
    v = random_field(op.n, 3)
    host_out = np.zeros_like(v)
    with Solver(links, dims, 0.12, nev=4, m=12, precision="fp64", k_max=1) as s:
        h = s._h
        st = lib().lqcd_apply(h, 0, 0, 1, C.c_void_p(v.ctypes.data), C.c_void_p(host_out.ctypes.data), 1)
        assert st == ERR_ARG
        tv = torch.from_numpy(v).to("cuda")
        tout = torch.zeros_like(tv)
        torch.cuda.synchronize()
        st = lib().lqcd_apply(h, 0, 0, 1, C.c_void_p(tv.data_ptr()), C.c_void_p(tout.data_ptr()), 0)
        assert st == ERR_ARG
        st = lib().lqcd_solve(h, 1, C.c_void_p(v.ctypes.data), C.c_void_p(host_out.ctypes.data), 1, 3, None)
        assert st == ERR_ARG
        tk = C.c_longlong()
        st = lib().lqcd_submit(h, C.c_void_p(tv.data_ptr()), C.c_void_p(host_out.ctypes.data), 1, 3, C.byref(tk))
        assert st == ERR_ARG
        ref = op.apply(v)
        assert np.abs(s.apply(v)[0] - ref).max() <= 1e-14 * np.abs(ref).max()


def test_apply_full_size_24x24x24x64_sampled():
    """The largest workload (10.6M unknowns): every site of a random field, FP64 and FP32."""
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload("24^3x64")
    v = random_field(op.n, 11)
    ref = op.apply(v)
    with Solver(links, w["dims"], w["kappa"], nev=4, m=12, precision="mixed", k_max=1) as s:
        out = s.apply(v)[0]
        assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()
        out32 = s.apply(v, precision="mixed")[0]
        assert rel(out32, ref) <= 2e-6


def test_operator_pair_full_size_autotuned_batch():
    """The launch configuration the benchmark times: 24^3x64, a batch of 8 slots,
    the operator-pair shape the autotuner picks. Slots 0 and 7 hold independent
    random fields, compared with the oracle's A and A^+ element by element
    (FP32 fields: 2e-6) with sigma = (phat, A p); slots 1..6 hold complex
    multiples of slot 0's fields, so their outputs must be the same multiples of
    slot 0's (a slot reading or writing another slot's data fails this)."""
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload("24^3x64")
    p0, p7 = random_field(op.n, 21), random_field(op.n, 27)
    h0, h7 = random_field(op.n, 41), random_field(op.n, 47)
    c = np.exp(1j * np.arange(1, 7)) * np.arange(2, 8) / 4.0
    p = np.stack([p0] + [ci * p0 for ci in c] + [p7])
    ph = np.stack([h0] + [ci * h0 for ci in c] + [h7])
    with Solver(links, w["dims"], w["kappa"], nev=4, m=12, precision="mixed", k_max=8) as s:
        shape = s.dslash_variant()
        ap, ahp, sig = s.apply_pair(p, ph, shape)
    del p, ph
    for i, (pi, hi) in ((0, (p0, h0)), (7, (p7, h7))):
        ref, refd = op.apply(pi), op.apply_dag(hi)
        assert rel(ap[i], ref) <= 2e-6, (shape, i)
        assert rel(ahp[i], refd) <= 2e-6, (shape, i)
        sref = np.vdot(hi, ref)
        assert abs(sig[i] - sref) <= 1e-5 * abs(sref), (shape, i)
    for j, ci in enumerate(c, start=1):
        assert rel(ap[j], ci * ap[0]) <= 1e-6, (shape, j)
        assert rel(ahp[j], ci * ahp[0]) <= 1e-6, (shape, j)
        assert abs(sig[j] - abs(ci) ** 2 * sig[0]) <= 1e-5 * abs(ci) ** 2 * abs(sig[0]), (shape, j)


@pytest.mark.parametrize("name", ["8^4", "16^3x32"])
def test_operator_pair_kernels_match_oracle(name):
    """Every shape of the BiCG operator-pair kernel (the autotuner's candidates:
    per-site and site-group thread maps, linear and brick site orders, and the TMA
    plane-streaming one, and the t-march brick orders): A p, A^+ phat and
    sigma = (phat, A p) against the oracle,
    FP32 fields, batches of 1 and 3."""
    from paper_0911_2285_gb300 import Solver
    w, links, op = workload(name)
    with Solver(links, w["dims"], w["kappa"], nev=1, m=3, precision="mixed", k_max=3, n_def_max=1) as s:
        for k in (1, 3):
            p = np.stack([random_field(op.n, 20 + i) for i in range(k)])
            ph = np.stack([random_field(op.n, 40 + i) for i in range(k)])
            refs = [(op.apply(p[i]), op.apply_dag(ph[i])) for i in range(k)]
            for variant in list(range(30)) + [100]:
                ap, ahp, sig = s.apply_pair(p, ph, variant)
                for i in range(k):
                    assert rel(ap[i], refs[i][0]) <= 2e-6, (variant, i)
                    assert rel(ahp[i], refs[i][1]) <= 2e-6, (variant, i)
                    sref = np.vdot(ph[i], refs[i][0])
                    assert abs(sig[i] - sref) <= 1e-5 * abs(sref), (variant, i)


def test_brick_shapes_rejected_on_small_extents():
    """Brick site orders need extents divisible by the brick's: refused on 4^4,
    not run (8 x 8 bricks, the 8 x 4 x 4 x 2 and 4 x 4 x 8 x 2 4-D bricks, the
    TMA-staged 8 x 4 x 4 x 2 bricks). The
    4^4 4-D brick covers the whole lattice, so every neighbour wraps into the
    block's own brick and every backward link comes from its face buffer."""
    from paper_0911_2285_gb300 import Solver, lqcd
    w, links, op = workload("4^4")
    with Solver(links, w["dims"], w["kappa"], nev=1, m=3, precision="mixed", k_max=2, n_def_max=1) as s:
        p = random_field(op.n, 1)
        for variant in (13, 14, 15, 19, 20, 21, 22, 23, 24, 26, 27, 28):
            with pytest.raises(lqcd.LQCDError):
                s.apply_pair(p, p, variant)
            with pytest.raises(lqcd.LQCDError):
                s.set_dslash_variant(variant)
        ph = random_field(op.n, 2)
        for variant in (2, 25, 29):
            ap, ahp, sig = s.apply_pair(np.stack([p, ph]), np.stack([ph, p]), variant)
            assert rel(ap[0], op.apply(p)) <= 2e-6 and rel(ap[1], op.apply(ph)) <= 2e-6
            assert rel(ahp[0], op.apply_dag(ph)) <= 2e-6 and rel(ahp[1], op.apply_dag(p)) <= 2e-6
            sref = np.vdot(ph, op.apply(p))
            assert abs(sig[0] - sref) <= 1e-5 * abs(sref)


@pytest.mark.parametrize("variant", [25, 26, 27])
def test_brick_shape_full_batch_solve(variant):
    """The 4-D brick shapes (every slot of the batch in one block; 26 stages
    links and spinor tiles in shared memory by TMA) in a full
    batch of 8 mixed-precision BiCG solves, pinned instead of the autotuner's
    pick: slots converge at different iterations, so later launches run with a
    partial mask of slots; every solution meets the FP64 residual with the
    oracle's operator, and the iteration counts match the per-slot shape's to
    FP32 rounding (+-2)."""
    from paper_0911_2285_gb300 import Solver
    from seeded_inputs import workload_source
    w, links, op = workload("8^4")
    b = np.stack([workload_source("8^4", 300 + i) for i in range(8)])
    b[3] *= 1e-3   # a scaled source: same iterations, different magnitudes in one batch
    b[5] = random_field(op.n, 77)
    kw = dict(nev=w["nev"], m=w["m"], n1=w["n1"], tol=1e-10, maxiter=2000, precision="mixed", k_max=8)
    with Solver(links, w["dims"], w["kappa"], **kw) as s:
        s.set_dslash_variant(2)
        _, ref, _ = s.solve(b, mode="plain")
        s.set_dslash_variant(variant)
        assert s.dslash_variant() == variant
        x, info, status = s.solve(b, mode="plain")
    assert status == 0
    for i in range(8):
        assert true_resid(op, b[i], x[i]) <= 1e-10, i
        assert abs(info[i]["iters"] - ref[i]["iters"]) <= 2, (i, info[i]["iters"], ref[i]["iters"])
    assert len({i["iters"] for i in info}) > 1
