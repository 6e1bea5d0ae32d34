"""Each planted mistake in the oracle (built with -DORACLE_MUTANT=k) must fail at least one pin.

The mistakes are the plausible ones: a min instead of the mean face opacity (Sec. 3.1), inward
edge normals (Eq. 2), a transposed rotation (Eq. 1), compositing with the transmittance after the
face instead of before it (Eq. 4), a dropped background term, integer instead of half-integer
pixel centres, a rotated barycentric index for depth, a flipped cross product in the pose
Jacobian (Eq. 7), a missing 1/(1 - alpha) in the adjoint, a descending depth sort, an
off-by-one tile box, a wrong loss normalisation; in the D-SSIM term of Eq. 8 the luminance
constant used for the contrast term, a dropped factor 2 in d(x^2)/dx, and edge clamping instead
of zero padding; and in the equilateral regulariser (Eq. 14) an angle measured between edges that
leave different vertices; and for the rendered normal map (Eq. 12) a normal left as the winding
gives it and a normal in world instead of camera space; and in the map statistics (Sec. 3.4) twice
the projected area and a coverage that also counts skipped contributions; and for the min-opacity
variant the mean's derivative under the minimum's value; and for the learnable-sigma variant a
derivative in sigma without the logarithm; and in the compositing of Eq. 4 a dropped alpha_max clamp, and a
walk that skips the face that would take T below T_min instead of stopping there.
"""
import pytest

import oracle_pins as P
from oracle.oracle import Oracle

MUTANTS = list(range(1, 25))


@pytest.mark.parametrize("k", MUTANTS)
def test_mutant_is_caught(k):
    o = Oracle(mutant=k)
    failed = []
    for pin in P.ALL_PINS:
        try:
            if pin is P.pin_fd_gradients:
                pin(o, seeds=(21,), sigmas=(1.0,))
            else:
                pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {k} passed every pin"
