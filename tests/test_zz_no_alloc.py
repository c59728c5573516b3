"""The allocation-free profile entry point, mpcd_profile_noalloc.

It is for callers that cannot allocate device memory when they ask for the
Poiseuille profile (services inside a fixed, pre-reserved device-memory
budget; job servers whose resident boxes fill the GPU's memory): it uses a
static 4096-bin device scratch array instead of allocating.  Checked here
through the C ABI against mpcd_profile, the entry point that allocates its
scratch, on two calls in a row (the shared array keeps the previous call's
contents, so the second call shows it is cleared), within the tolerance of
the other GPU tests.  The first call comes straight after stepping, so it
also completes the pending collision itself.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1801_10187_gb300 as pkg  # noqa: E402
from paper_1801_10187_gb300 import inputs  # noqa: E402

TOL = 1e-12


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_profile_noalloc_matches_profile_on_two_calls(precision):
    n = (6, 5, 12)
    s = inputs.solvent(n, 10, seed=17, mixed=precision == "mixed")
    box = pkg.Box(n=n, seed=17, precision=precision, thermostat=True, walls_z=True,
                  body_force=(0.02, 0.0, 0.0), virt_density=10.0)
    box.set_state(s.pos, s.vel)
    box.step(20)
    # the collision of the last step is still pending: the allocation-free
    # call completes it before it reads the state
    first = box.profile_noalloc(24)
    ref = box.profile(24)
    second = box.profile_noalloc(24)
    # a twin box stepped the same way, profiled by the allocating call alone
    twin = pkg.Box(n=n, seed=17, precision=precision, thermostat=True, walls_z=True,
                   body_force=(0.02, 0.0, 0.0), virt_density=10.0)
    twin.set_state(s.pos, s.vel)
    twin.step(20)
    np.testing.assert_allclose(first, twin.profile(24), rtol=0, atol=TOL)
    twin.close()
    np.testing.assert_allclose(first, ref, rtol=0, atol=TOL)
    np.testing.assert_allclose(second, ref, rtol=0, atol=TOL)
    # a smaller request after a larger one: nothing of the earlier call leaks in
    ref7 = box.profile(7)
    np.testing.assert_allclose(box.profile_noalloc(7), ref7, rtol=0, atol=TOL)
    np.testing.assert_allclose(box.profile_noalloc(7), ref7, rtol=0, atol=TOL)
    # the static scratch holds 4096 bins
    with pytest.raises(pkg.MpcdError) as e:
        box.profile_noalloc(4097)
    assert e.value.code == pkg.MPCD_EINVAL
    box.close()


def test_profile_noalloc_needs_the_box_on_the_device():
    n = (4, 4, 4)
    s = inputs.solvent(n, 5, seed=3)
    box = pkg.Box(n=n, seed=3, precision="fp64")
    box.set_state(s.pos, s.vel)
    with pytest.raises(pkg.MpcdError) as e:
        box.profile_noalloc(8)
    assert e.value.code == pkg.MPCD_ESTATE
    box.step(0)
    np.testing.assert_allclose(box.profile_noalloc(8), box.profile(8), rtol=0, atol=TOL)
    box.close()
