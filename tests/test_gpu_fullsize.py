"""The two largest contractions of the chi = 48, r = 3 step (Eqs. 6-7, C2 and C4) at their
full shapes, through tatrg_contract with the multi-mode strides the step uses, in each tile
form of the tensor-core path (single CTAs, CTA pairs, multicast clusters).  Inputs are seeded
normal operands drawn on the device; each of 2000 sampled outputs is checked against its
float64 dot product, formed on the host from the operand entries it sums."""
import numpy as np
import pytest

import paper_2412_14104_gb300 as tg
from paper_2412_14104_gb300 import synth

pytestmark = pytest.mark.gpu

# chi = 48, r = 3 steady state: D0 = Da = Ds = Dg = Ks = 48, KA = KX = r chi = 144, Kg = chi^2
D0 = Da = Ds = Dg = Ks = 48
KA = KX = 144
Kg = 48 * 48
NS = 2000
TOL = {tg.TF32X3: 5e-6, tg.BF16X3: 1e-4, tg.BF16X6: 5e-6, tg.OZAKI: 1e-8}  # as for the small contraction tests


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def _err(got, want):
    return np.max(np.abs(got - want)) / np.max(np.abs(want))


# (precision, tile form): -1 single CTAs, 1 CTA pairs, 2 multicast clusters (tatrg_set_cta_pairs)
FORMS = [(tg.TF32X3, -1), (tg.TF32X3, 1), (tg.TF32X3, 2), (tg.BF16X3, -1), (tg.BF16X3, 2),
         (tg.BF16X6, -1), (tg.BF16X6, 2), (tg.OZAKI, 0)]


@pytest.fixture
def form(request):
    tg.set_cta_pairs(request.param)
    yield request.param
    tg.set_cta_pairs(0)


@pytest.mark.parametrize("prec,form", FORMS, indirect=["form"])
def test_c2_full_shape_sampled(torch, prec, form):
    """C2: q[i0,kA,k,kX,g] = sum_{a,b} em[i0,kA,a,b,k] F[a,kX,b,g];
    M = 331776, N = 6912, K = 2304 (18 GB float64 output)."""
    em = synth.device_normal(41, (D0 * KA, Da, Ds, Ks))
    F = synth.device_normal(42, (Da, KX, Ds, Dg))
    q = torch.empty((D0 * KA, Ks, KX, Dg), dtype=torch.float64, device="cuda")
    m = [(D0 * KA, Da * Ds * Ks, Ks * KX * Dg), (Ks, 1, KX * Dg)]
    n = [(KX, Ds * Dg, Dg), (Dg, 1, 1)]
    k = [(Da, Ds * Ks, KX * Ds * Dg), (Ds, Ks, Dg)]
    tg.contract(m, n, k, em, F, q, precision=prec)
    torch.cuda.synchronize()
    rng = np.random.default_rng(43)
    r_ik = rng.integers(0, D0 * KA, NS)
    r_k = rng.integers(0, Ks, NS)
    c_x = rng.integers(0, KX, NS)
    c_g = rng.integers(0, Dg, NS)
    dev = lambda a: torch.from_numpy(a).cuda()
    rows = em[dev(r_ik), :, :, dev(r_k)].reshape(NS, -1).cpu().numpy()      # [s, (a, b)]
    cols = F[:, dev(c_x), :, dev(c_g)].reshape(NS, -1).cpu().numpy()   # [s, (a, b)]
    want = np.einsum("sj,sj->s", rows, cols)
    got = q[dev(r_ik), dev(r_k), dev(c_x), dev(c_g)].cpu().numpy()
    del em, F, q
    torch.cuda.empty_cache()
    print("precision %d form %d: max relative error %.3e" % (prec, form, _err(got, want)))
    assert _err(got, want) < TOL[prec], _err(got, want)


@pytest.mark.parametrize("prec,form", FORMS, indirect=["form"])
def test_c4_full_shape_sampled(torch, prec, form):
    """C4: out[i0,kG,k,g] = sum_{kA,kX} q[i0,kA,k,kX,g] P[kA,kX,kG];
    M = 110592, N = 2304, K = 20736 (the 18 GB intermediate q as operand)."""
    q = synth.device_normal(44, (D0, KA, Ks, KX, Dg))
    P = synth.device_normal(45, (KA, KX, Kg))
    out = torch.empty((D0, Kg, Ks, Dg), dtype=torch.float64, device="cuda")
    m = [(D0, KA * Ks * KX * Dg, Kg * Ks * Dg), (Ks, KX * Dg, Dg), (Dg, 1, 1)]
    n = [(Kg, 1, Ks * Dg)]
    k = [(KA, Ks * KX * Dg, KX * Kg), (KX, Dg, Kg)]
    tg.contract(m, n, k, q, P, out, precision=prec)
    torch.cuda.synchronize()
    rng = np.random.default_rng(46)
    r_i = rng.integers(0, D0, NS)
    r_k = rng.integers(0, Ks, NS)
    r_g = rng.integers(0, Dg, NS)
    c_u = rng.integers(0, Kg, NS)
    dev = lambda a: torch.from_numpy(a).cuda()
    rows = q[dev(r_i), :, dev(r_k), :, dev(r_g)].reshape(NS, -1).cpu().numpy()   # [s, (kA, kX)]
    cols = P[:, :, dev(c_u)].permute(2, 0, 1).reshape(NS, -1).cpu().numpy()
    want = np.einsum("sj,sj->s", rows, cols)
    got = out[dev(r_i), dev(c_u), dev(r_k), dev(r_g)].cpu().numpy()
    del q, P, out
    torch.cuda.empty_cache()
    print("precision %d form %d: max relative error %.3e" % (prec, form, _err(got, want)))
    assert _err(got, want) < TOL[prec], _err(got, want)
