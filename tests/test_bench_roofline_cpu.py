"""The per-element algorithmic flops and bytes that bench.py divides by the
measured kernel times (the roofline's `achieved`), checked against counts
written out term by term: the three stages of Algorithm 2 (Sec. 3.2) with
the last one over the symmetric half of the element matrix, and the output,
coefficient, geometry and dof-map bytes."""
import bench


def _sf_flops_3d(p, q, stiffness_terms, mass, x_patterns):
    """Multiply-add = 2 flops.  Stage 1 contracts k3 for every (k1, k2) and
    every (a3, b3) pair: n^2 q^3 multiply-adds per term; stage 2 contracts k2
    for every k1, (a2, b2) and (a3, b3): n^4 q^2 per term; stage 3 contracts
    k1 for every entry of the symmetric half, once per x pattern."""
    n = p + 1
    N = n ** 3
    S = N * (N + 1) // 2
    fma = 0
    for _ in range(stiffness_terms):
        fma += n * n * q ** 3 + n ** 4 * q * q
    if stiffness_terms:
        fma += x_patterns * q * S
    if mass:
        fma += n * n * q ** 3 + n ** 4 * q * q + q * S
    return 2 * fma


def test_flops_per_element():
    # identity map: three diagonal stiffness terms, x patterns 11 and 00
    assert bench.flops_per_element(3, 3, 4, True, True, False) == _sf_flops_3d(3, 4, 3, True, 2) == 90880
    # general map: nine terms, four x patterns (11, 00, 10, 01)
    assert bench.flops_per_element(3, 4, 5, True, False, True) == _sf_flops_3d(4, 5, 9, False, 4) == 652500
    assert bench.flops_per_element(3, 8, 9, True, True, False) == _sf_flops_3d(8, 9, 3, True, 2) == 19092510


def test_classical_flops_per_element():
    # every entry of the symmetric half at every Gauss point: d gradient
    # products for the stiffness, one product for the mass
    N, Q = 64, 64
    assert bench.classical_flops_per_element(3, 3, 4, True, True) == 2 * (N * (N + 1) // 2) * Q * 4


def test_bytes_per_element():
    # K and M in FP64, kappa per point, the dof map (int32)
    assert bench.bytes_per_element(3, 3, 4, 8, True, True, False) == 64 * 64 * 8 * 2 + 64 * 8 + 64 * 4 == 66304
    # curved p = 4 stiffness in FP32: kappa and the 3 x 3 Jacobian per point in FP64
    assert bench.bytes_per_element(3, 4, 5, 4, True, False, True) == 125 * 125 * 4 + 125 * 8 + 125 * 72 + 125 * 4 == 73000
    assert bench.bytes_per_element(3, 5, 6, 4, True, True, False) == 216 * 216 * 4 * 2 + 216 * 8 + 216 * 4 == 375840
    assert bench.bytes_per_element(3, 8, 9, 8, True, True, False) == 729 * 729 * 8 * 2 + 729 * 8 + 729 * 4 == 8511804
