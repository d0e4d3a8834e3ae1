"""The C-ABI library loads and exports every entry point include/rcp.h declares
(no compute call: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rcp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_12235_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "rcp_create" in names and "rcp_run" in names and "rcp_energy_grad" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2608_12235_b300 import rcp
    assert sorted(rcp.EXPORTS) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_2608_12235_b300 import rcp
    rcp.load()
    cfg = rcp.rcp_config_default()
    assert cfg.tol == 5e-4 and (cfg.Y, cfg.X) == (2, 9) and cfg.beta1 == 0.9 and cfg.beta2 == 0.999
    assert rcp.load().rcp_status_str(2).decode().startswith("periodic-image")


def test_create_rejects_bad_input_before_touching_the_gpu(lib):
    from paper_2608_12235_b300 import rcp
    import numpy as np
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_create(np.array([1.0, -1.0]), 1.0, 0)
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_create(np.ones(4), np.ones(4), 0, d=4)   # d is 2 or 3
    assert e.value.status == 9


def test_seated_and_cascade_reject_bad_input_before_touching_the_gpu(lib):
    from paper_2608_12235_b300 import rcp
    import numpy as np
    with pytest.raises(rcp.RcpError) as e:   # one wall bit per axis of the caller
        rcp.rcp_create_seated([1.0], [[0.5, 0.5, 0.5]], [1.0], 1.0, 0, rcp.rcp_config_default(walls=8))
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:   # a frozen diameter must be positive
        rcp.rcp_create_seated([-1.0], [[0.5, 0.5, 0.5]], [1.0], 1.0, 0)
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:   # a frozen position must be finite
        rcp.rcp_create_seated([1.0], [[0.5, np.nan, 0.5]], [1.0], 1.0, 0)
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:   # class 1 is empty
        rcp.rcp_cascade([1.0, 1.0], [0, 2])
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:   # no such container, whatever the call
        rcp.rcp_cascade([1.0, 1.0], [0, 1], cfg=rcp.rcp_config_default(container=3, precision=rcp.RCP_MIXED))
    assert e.value.status == 1


def test_walls_are_checked_before_touching_the_gpu(lib):
    from paper_2608_12235_b300 import rcp
    import numpy as np
    with pytest.raises(rcp.RcpError) as e:   # one bit per axis, either precision
        rcp.rcp_create(np.ones(4), 1.0, 0, rcp.rcp_config_default(precision=rcp.RCP_MIXED, walls=8))
    assert e.value.status == 1
    with pytest.raises(rcp.RcpError) as e:   # no z axis when d = 2
        rcp.rcp_create(np.ones(4), 1.0, 0, rcp.rcp_config_default(walls=4), d=2)
    assert e.value.status == 1


def test_container_is_checked_before_touching_the_gpu(lib):
    from paper_2608_12235_b300 import rcp
    import numpy as np
    for cfg, d, want in [(rcp.rcp_config_default(container=3), 3, 1),
                         (rcp.rcp_config_default(container=2), 2, 1),   # a cylinder needs z
                         (rcp.rcp_config_default(container=-1, precision=rcp.RCP_MIXED), 3, 1)]:
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_create(np.ones(4), 1.0, 0, cfg, d=d)
        assert e.value.status == want
