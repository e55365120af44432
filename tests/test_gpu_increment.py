"""The FP32 phase in increment form (X = X_b + delta) on blocks of the width
for which the pipelined tall-skinny kernels run (32 < p <= 64, like the
64^3 x 64 system): the two Grams of dS in one pass (pair form), D^T M D and
X^T M D with M D read once (shared form), and the three-term retraction
update that also forms the trial's density.  Compared with the FP64
oracle's trajectory (Alg. ConOptM, Sec. 3) and with the oracle's energy of
the returned block (Sec. 2.3)."""
import numpy as np
import pytest

import ks_inputs as ki
from oracle import energy as oe
from oracle import stiefel as ost

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# p = 36: 9 float4 columns of a 64-wide tile, the rest of the tile padding;
# n = 14^3 = 2744 leaves a ragged last row tile and a ragged last row stage
CASE = dict(N=14, L=8.0, natoms=4, p=36, Z=4.0, seed=11)
ITERS = 12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("tensor_cores", [1, 3], ids=["simt_updates", "tc_updates"])
@pytest.mark.parametrize("retraction", ["qr", "cayley"])
def test_increment_form_on_a_wide_block_follows_fp64(retraction, tensor_cores):
    # tensor_cores 3 runs the narrow updates on the tensor cores (three TF32
    # products per term), 1 on the FP32 pipes
    import paper_1308_2864_gb300 as ks
    s = ki.small_system(**CASE)
    model = oe.Model.from_system(s)
    ref = ost.minimize(model, s.x0(), ost.Options(retraction=retraction, maxit=ITERS))
    P = ks.Problem.from_system(s)
    P.set_tensor_cores(tensor_cores)
    X = dev(s.x0())
    r = P.minimize(X, retraction=retraction, gtol=1e-12, maxit=ITERS, precision="mixed",
                   stall_iters=0)
    assert r["mixed_iters"] == ITERS and r["status"] == ks.KS_ENOCONV
    Xh = X.cpu().numpy()
    # the energy the increment form reports is that of the block it returns
    # (its density came from the retraction's update pass).  Twelve
    # iterations from the start stay below the first refresh of the base, so
    # delta is as large as X itself and the FP32 increments carry ~1e-7 of
    # each energy term (the total can be far smaller than its terms); an
    # indexing error in any of the kernels moves it by far more than the
    # 1e-6 of the terms allowed here.
    ev = oe.evaluate(model, Xh)
    scale = sum(abs(v) for v in ev.parts.values())
    assert abs(r["E"] - ev.E) <= 1e-6 * scale
    # and the iterates follow the FP64 trajectory (the early BB steps
    # amplify the update's rounding, about eight times larger with three
    # TF32 products than on the FP32 pipes)
    assert abs(r["E"] - ref.E) <= (1e-6 if tensor_cores == 1 else 1e-5) * scale
    assert r["gradnorm"] == pytest.approx(ref.dnorm, rel=1e-3)
    # the trial keeps X^T M X - I of the iterate (exact trial Gram) up to the
    # rounding of the update: about 1e-7 relative per product on the FP32
    # pipes, 2^-21 with three TF32 products, over twelve steps of the size of
    # X; an indexing error gives O(1)
    assert ost.ortho_error(model, Xh) < (1e-6 if tensor_cores == 1 else 1e-4)
