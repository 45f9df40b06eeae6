"""Host side of the learned preconditioner's training driver: the flat
parameter layout (nn.layer_shapes) agrees layer by layer with the one the
oracle's network reads, and nn.init_params draws He-normal weights and zero
biases in that layout."""
import numpy as np
import pytest

from oracle import unet as ou
from paper_1301_3925_gb300 import nn


@pytest.mark.parametrize("c", [(16, 32, 64), (8, 12, 20)])
def test_layer_layout_matches_oracle(c):
    mine = nn.layer_shapes(nn.NF, *c)
    theirs = [(co, ci, k) for _, co, ci, k in ou.layer_shapes(nn.NF, c1=c[0], c2=c[1], c3=c[2])]
    assert mine == theirs
    assert sum(co * ci * k * k + co for co, ci, k in mine) == ou.n_params(nn.NF, c1=c[0], c2=c[1], c3=c[2])


def test_init_params_he_normal_zero_bias():
    shapes = nn.layer_shapes(nn.NF, 16, 32, 64)
    P = sum(co * ci * k * k + co for co, ci, k in shapes)
    th = nn.init_params(P, shapes, 7)
    assert th.dtype == np.float32 and th.shape == (P,)
    assert np.array_equal(th, nn.init_params(P, shapes, 7))
    o = 0
    for co, ci, k in shapes:
        nw = co * ci * k * k
        w, b = th[o:o + nw], th[o + nw:o + nw + co]
        o += nw + co
        assert np.all(b == 0.0)
        std = np.sqrt(2.0 / (ci * k * k))
        if nw >= 1000:   # enough draws for a statistical check
            assert abs(w.std() / std - 1.0) < 0.1 and abs(w.mean()) < 0.1 * std
    assert o == P
    with pytest.raises(AssertionError):
        nn.init_params(P + 1, shapes, 7)


def test_constants():
    # 16 residual values of a 4 x 4 block plus 9 stencil means
    assert nn.RF == 4 and nn.NF == nn.RF * nn.RF + 9
