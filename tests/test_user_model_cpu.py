"""Host logic of user-defined models (sdeb_create_user), no GPU needed: the
run-time compiler checks the source on the host, so a source that does not
compile is refused with the compiler's message; argument validation."""
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

import user_models


@pytest.fixture(scope="module", autouse=True)
def _built():
    sdeb_build.build()
    sdeb.lib()


def _pb(n=2, m=3, d=10, **kw):
    return sdeb.Problem.make("user", n, 4, 0.01, 10, 5, 1, "fp64", m=m, d=d, **kw)


def test_a_source_that_does_not_compile_is_refused_with_the_log():
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create_user(_pb(), user_models.BROKEN)
    if e.value.status == sdeb.SDEB_EUNSUPPORTED:
        pytest.skip("libnvrtc is not available on this host")
    assert e.value.status == sdeb.SDEB_EINVAL
    assert "undefined_symbol_here" in str(e.value) and "user_model" in str(e.value)


def test_a_valid_source_compiles():
    try:
        ctx = sdeb.sdeb_create_user(_pb(), user_models.LINEAR_DENSE)
    except sdeb.SdebError as e:
        if e.status == sdeb.SDEB_EUNSUPPORTED:
            pytest.skip("libnvrtc is not available on this host")
        assert e.status == sdeb.SDEB_ECUDA     # compiled; no device to load it on
        assert "loading the compiled kernel" in str(e)
    else:
        sdeb.sdeb_destroy(ctx)


def test_user_problem_validation():
    import ctypes
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create(_pb())                                      # needs the source
    assert e.value.status == sdeb.SDEB_EINVAL
    for bad, status in ((_pb(n=65, m=1, d=1), sdeb.SDEB_EINVAL), (_pb(m=65), sdeb.SDEB_EINVAL),
                        (_pb(milstein=True), sdeb.SDEB_EUNSUPPORTED),
                        (_pb(implicit="euler"), sdeb.SDEB_EUNSUPPORTED),
                        (_pb(implicit="midpoint"), sdeb.SDEB_EUNSUPPORTED),
                        (_pb(ckpt_every=5), sdeb.SDEB_EUNSUPPORTED)):
        with pytest.raises(sdeb.SdebError) as e:
            sdeb.sdeb_create_user(bad, user_models.LINEAR_DENSE)
        assert e.value.status == status
    ctx = ctypes.c_void_p()
    assert sdeb.lib().sdeb_create_user(ctypes.byref(_pb()), None, ctypes.byref(ctx)) == sdeb.SDEB_EINVAL
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create_user(sdeb.Problem.make("ou", 2, 4, 0.01, 10, 5, 1, "fp64"), user_models.LINEAR_DENSE)
    assert e.value.status == sdeb.SDEB_EINVAL
