"""Algorithmic bytes per node-step that bench.py divides by, checked against
a count written out here: read and write of the 8N moving populations (eight
per order parameter and eight of g), the N - 1 rest slots, phi_i(t-1) and
u(t-1), plus p(t-1) for the 16-bit forms."""
import pytest

import bench


@pytest.mark.parametrize("N", [3, 4, 5])
@pytest.mark.parametrize("prec,s_mov,s_state,extra", [
    ("fp64", 8, 8, 0), ("fp32", 4, 4, 0), ("bf16", 2, 4, 1), ("fp16", 2, 4, 1)])
def test_alg_bytes_per_node(N, prec, s_mov, s_state, extra):
    moving = 8 * (N - 1) + 8
    state = (N - 1) + (N - 1) + 2 + extra
    assert bench.alg_bytes_per_node(N, prec) == 2 * (moving * s_mov + state * s_state)


def test_headline_figures():
    assert bench.alg_bytes_per_node(5, "fp32") == 400
    assert bench.alg_bytes_per_node(5, "bf16") == 248
    assert bench.alg_bytes_per_node(5, "fp64") == 800
