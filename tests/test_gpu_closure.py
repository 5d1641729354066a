"""Learned-closure kernels against the FP64 reference (oracle/closure.py)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from oracle import closure as C  # noqa: E402
from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import closure as CL  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402
from paper_2011_06856_gb300 import workloads as W  # noqa: E402

B.build()
N, K, KF = 2, 24, 128


def bf16(a):
    """Round to BF16 (nearest even), as the device copy of the weights."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def ref_params(cl):
    p = cl.split_params(cl.get_params().astype(np.float64))
    return [bf16(p[0]), p[1], bf16(p[2]), p[3], bf16(p[4]), p[5]]


def random_coarse_populations(sites, seed, n=N, k=K):
    q = O.Quadrature(n, k)
    g = np.random.default_rng(seed)
    f = np.stack([q.feq(g.uniform(0.3, 1), g.uniform(0.5, 1.1), g.uniform(-0.2, 0.2),
                        g.uniform(-0.2, 0.2)) for _ in range(sites)], axis=1)
    f *= g.uniform(0.9, 1.1, f.shape)  # off equilibrium
    return q, f


def test_features_restriction_target_match_reference():
    cl = R.Closure(N, K, seed=1)
    q, f = random_coarse_populations(300, 0)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    X = torch.zeros((cl.F, 300), dtype=torch.float32, device="cuda")
    cl.features(fd, 0.37, X)
    cl.stream.synchronize()
    ref = C.features(f.astype(np.float32).astype(np.float64), q.p0, q.vx, q.vy, q.w, 0.37).T
    np.testing.assert_allclose(X.cpu().numpy(), ref, rtol=2e-5, atol=2e-6)
    # restriction of fine populations
    qf = O.Quadrature(N, KF)
    ff = np.random.default_rng(4).uniform(0.1, 1, (qf.npop, 50)) * qf.w[:, None]
    ffd = torch.tensor(ff, dtype=torch.float32, device="cuda")
    fcd = torch.zeros((cl.npop, 50), dtype=torch.float32, device="cuda")
    cl.restrict(KF, ffd, fcd)
    np.testing.assert_allclose(fcd.cpu().numpy(), C.restrict(ff.astype(np.float32).astype(np.float64), N, KF, K),
                               rtol=2e-5, atol=1e-9)
    # target
    T = torch.zeros((cl.npop, 50), dtype=torch.float32, device="cuda")
    fc2 = fcd * 1.01
    cl.target(fcd, fc2, T)
    cl.stream.synchronize()
    a, b = fcd.double().cpu().numpy(), fc2.double().cpu().numpy()
    n0 = q.p0 @ b
    np.testing.assert_allclose(T.cpu().numpy(), (a - b) / (q.w[:, None] * n0[None, :]), rtol=1e-4, atol=1e-6)


def test_forward_and_gradient_match_reference():
    cl = R.Closure(N, K, seed=2)
    g = np.random.default_rng(5)
    S = 700
    X = g.normal(0, 0.5, (cl.F, S)).astype(np.float32)
    T = g.normal(0, 0.1, (cl.npop, S)).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    Y = torch.zeros((cl.npop, S), dtype=torch.float32, device="cuda")
    cl.forward(Xd, 0, S, Y)
    cl.stream.synchronize()
    params = ref_params(cl)
    yref, _ = C.mlp_forward(params, X.T.astype(np.float64))
    np.testing.assert_allclose(Y.cpu().numpy(), yref.T, rtol=1e-4, atol=1e-5)
    work = cl.work(S)
    cl.set_train_path(False)  # one thread per site, FP32 activations and deltas
    grad, loss = cl.gradient(Xd, Td, 100, 500, work)
    lref, gref = C.mlp_loss_and_grad(params, X[:, 100:600].T.astype(np.float64),
                                     T[:, 100:600].T.astype(np.float64))
    assert abs(loss - lref) < 1e-4 * lref
    flat = np.concatenate([a.ravel() for a in gref])
    assert np.abs(grad - flat).max() < 1e-3 * np.abs(flat).max()


def bf16_loss_and_grad(params, X, T):
    """Loss and gradient with the BF16 roundings of the tensor-core training
    kernel: the layer inputs x, h1, h2 and the deltas dY, dz2, dz1 rounded to
    BF16 where they enter a product (bias gradients from the unrounded deltas);
    FP64 otherwise."""
    W1, b1, W2, b2, W3, b3 = params
    xb = bf16(X)
    z1 = xb @ W1 + b1
    h1 = bf16(C.gelu(z1))
    z2 = h1 @ W2 + b2
    h2 = bf16(C.gelu(z2))
    y = h2 @ W3 + b3
    dY = 2.0 * (y - T) / y.size
    dYb = bf16(dY)
    dz2 = (dYb @ W3.T) * C.gelu_grad(z2)
    dz2b = bf16(dz2)
    dz1 = (dz2b @ W2.T) * C.gelu_grad(z1)
    dz1b = bf16(dz1)
    g = (xb.T @ dz1b, dz1.sum(0), h1.T @ dz2b, dz2.sum(0), h2.T @ dYb, dY.sum(0))
    return float(((y - T) ** 2).mean()), g


@pytest.mark.parametrize("n,k,S,off,count", [(2, 24, 700, 100, 500), (2, 24, 21000, 300, 20000),
                                             (2, 16, 1500, 0, 1333), (3, 16, 1500, 17, 1400)])
def test_tensor_core_gradient_matches_bf16_reference(n, k, S, off, count):
    """Fused tensor-core training pass (ragged last tile; above 152 x 128
    columns the CTAs loop over tiles) against the reference with the same BF16
    roundings, and against the exact FP64 gradient: the BF16 roundings of the
    activations and deltas (relative 2^-9) leave the gradient direction intact."""
    cl = R.Closure(n, k, seed=11)
    g = np.random.default_rng(n * 100 + k)
    X = g.normal(0, 0.5, (cl.F, S)).astype(np.float32)
    T = g.normal(0, 0.1, (cl.npop, S)).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    cl.set_train_path(True)
    grad, loss = cl.gradient(Xd, Td, off, count, cl.work(S))
    params = ref_params(cl)
    Xs = X[:, off:off + count].T.astype(np.float64)
    Ts = T[:, off:off + count].T.astype(np.float64)
    lb, gb = bf16_loss_and_grad(params, Xs, Ts)
    flat = np.concatenate([a.ravel() for a in gb])
    assert abs(loss - lb) < 1e-4 * lb
    assert np.abs(grad - flat).max() < 2e-3 * np.abs(flat).max()
    lref, gref = C.mlp_loss_and_grad(params, Xs, Ts)
    exact = np.concatenate([a.ravel() for a in gref])
    assert abs(loss - lref) < 1e-2 * lref
    cos = float(grad @ exact / (np.linalg.norm(grad) * np.linalg.norm(exact)))
    assert cos > 0.999, cos


def bf16_forward(params, X):
    """The network with its layer inputs rounded to BF16, as the tensor-core kernel
    feeds them (features, GELU outputs); FP64 otherwise."""
    W1, b1, W2, b2, W3, b3 = params
    h1 = bf16(C.gelu(bf16(X) @ W1 + b1))
    h2 = bf16(C.gelu(h1 @ W2 + b2))
    return h2 @ W3 + b3


def apply_case(sites, seed, tensor_cores, n=N, k=K, ref_bf16=None):
    """Apply the correction to random off-equilibrium populations through the
    chosen kernel (the tensor-core one falls back to the other for rules it has
    no specialisation for); returns the reference next to the result."""
    ref_bf16 = tensor_cores if ref_bf16 is None else ref_bf16
    cl = R.Closure(n, k, seed=3)
    cl.set_apply_path(tensor_cores)
    q, f = random_coarse_populations(sites, seed, n, k)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda").contiguous()
    f32 = fd.double().cpu().numpy()
    cl.apply_buffer(fd.data_ptr(), sites, 0.3)
    cl.stream.synchronize()
    got = fd.double().cpu().numpy()
    # reference: features -> network -> denormalise -> projection -> add
    params = ref_params(cl)
    X = C.features(f32, q.p0, q.vx, q.vy, q.w, 0.3)
    y = bf16_forward(params, X) if ref_bf16 else C.mlp_forward(params, X)[0]
    n0 = q.p0 @ f32
    d = y.T * q.w[:, None] * n0[None, :]
    ref = f32 + C.conservative_projection(d, q.p0, q.vx, q.vy, q.w)
    Cm = np.stack([q.p0, q.p0 ** 2, q.p0 ** 2 * q.vx, q.p0 ** 2 * q.vy])
    return q, f32, got, ref, d, Cm


@pytest.mark.parametrize("n,k", [(2, 24), (2, 20)])
def test_apply_conserves_and_matches_reference(n, k):
    """One thread per site, FP32 activations: FP32 rounding only.  (2, 20) has no
    tensor-core specialisation (60 populations) and takes this kernel by default."""
    q, f32, got, ref, d, Cm = apply_case(333, 6, k == 20, n, k, ref_bf16=False)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-7 * np.abs(f32).max())
    before, after = Cm @ f32, Cm @ got
    assert np.abs(after - before).max() < 2e-6 * np.abs(before).max()


@pytest.mark.parametrize("n,k,sites", [(2, 24, 16), (2, 24, 333), (2, 24, 5000), (2, 24, 40000),
                                       (2, 24, 45001), (2, 16, 3001), (3, 16, 4000)])
def test_apply_tensor_cores_conserves_and_matches_reference(n, k, sites):
    """BF16 mma.sync path (192-site CTA tiles; ragged last tile; site counts that
    are not a multiple of 4 take the 4-byte copy form; above 152 x 192 sites the
    CTAs loop over tiles through both population buffers; the conservative
    projection folded into the last layer) against the reference with the same
    BF16 roundings of the layer inputs.  A rare flip of one BF16 rounding (FP32
    vs FP64 sums on either side of a rounding boundary) moves an output by about
    a BF16 ulp of one activation times a weight, hence the absolute term in
    units of the correction."""
    q, f32, got, ref, d, Cm = apply_case(sites, 6 + sites, True, n, k)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-3 * np.abs(d).max())
    med = np.median(np.abs(got - ref)) / np.abs(d).max()
    assert med < 1e-4
    before, after = Cm @ f32, Cm @ got
    assert np.abs(after - before).max() < 2e-6 * np.abs(before).max()


def test_training_on_method_data_reduces_loss():
    cl = R.Closure(N, K, seed=4)
    X, T = CL.generate(cl, 32, KF, kns=(0.05, 0.5), steps=12)
    assert X.shape[1] == 2 * 12 * 32 * 32
    assert torch.isfinite(X).all() and torch.isfinite(T).all()
    losses = CL.train(cl, X, T, iters=120, batch=2048, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5]), (losses[:5], losses[-20:])


def test_trained_closure_reduces_coarse_error_vs_fine():
    """Gain test: trained on runs of the method itself (K = 128 fine, K = 24 coarse;
    tensor-core training, 4000 Adam steps of 16384 columns, cosine step decay),
    the corrected coarse run is closer to the fine run than the plain coarse run
    (relative L2, Eq. rel_err, of n and eps) on a Riemann problem not in the
    training set, at Kn = 0.3 and Kn = 1."""
    cl = R.Closure(N, K, seed=7)
    X, T = CL.generate(cl, 64, KF, kns=(0.02, 0.1, 0.5, 2.0), steps=48, every=2)
    CL.train(cl, X, T, iters=4000, batch=16384, lr=2e-3, decay=True)
    plain, learned = [], []
    for kn in (0.3, 1.0):
        mf, mc, ml = CL.deploy(cl, 64, KF, kn, 48)
        for i in (0, 1):
            plain.append(CL.rel_l2(mc[i], mf[i]))
            learned.append(CL.rel_l2(ml[i], mf[i]))
    print("plain", plain, "learned", learned)
    assert np.mean(learned) < 0.8 * np.mean(plain)


def test_apply_tensor_cores_full_size_4096sq_sampled():
    """The deployed correction at the learned-closure benchmark size (4096^2
    coarse sites, 72 populations, FP32; one persistent CTA per SM looping over
    about 575 tiles each): a block of 4096 random off-equilibrium sites, repeated
    over the grid on the device, corrected in place; 2000 sampled sites checked
    against the BF16-rounding reference of their block site."""
    n, blk = 4096, 4096
    S = n * n
    cl = R.Closure(N, K, seed=3)
    q, f = random_coarse_populations(blk, 21)
    f32 = f.astype(np.float32)
    fd = torch.tensor(f32, device="cuda").repeat(1, S // blk).contiguous()
    torch.cuda.synchronize()  # the repeat ran on torch's stream; the correction runs on the closure's
    cl.apply_buffer(fd.data_ptr(), S, 0.3)
    cl.stream.synchronize()
    idx = np.sort(np.random.default_rng(5).choice(S, 2000, replace=False))
    got = fd[:, torch.tensor(idx, device="cuda")].double().cpu().numpy()
    del fd
    params = ref_params(cl)
    fb = f32.astype(np.float64)
    X = C.features(fb, q.p0, q.vx, q.vy, q.w, 0.3)
    y = bf16_forward(params, X)
    n0 = q.p0 @ fb
    d = y.T * q.w[:, None] * n0[None, :]
    ref = (fb + C.conservative_projection(d, q.p0, q.vx, q.vy, q.w))[:, idx % blk]
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=2e-3 * np.abs(d).max())
    assert np.median(np.abs(got - ref)) / np.abs(d).max() < 1e-4
