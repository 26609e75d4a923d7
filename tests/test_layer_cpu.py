"""Host-side logic of the torch wrappers (no GPU): option selection and the
shape rules for grey guides and the per-resolution transform."""
import pytest
import torch

from paper_1803_05619_gb300 import layer


def test_default_calls_need_no_options():
    assert layer._options(True, 3, torch.empty(1, 3, 8, 8), None) is None


def test_grey_guide_option():
    opt = layer._options(True, 1, torch.empty(1, 3, 8, 8), None)
    assert (opt.mean_ab, opt.guide_channels, opt.guide_low) == (1, 3, 0)
    opt = layer._options(False, 2, torch.empty(1, 2, 8, 8), None)
    assert (opt.mean_ab, opt.guide_channels, opt.guide_low) == (0, 0, 0)


def test_guide_low_needs_the_transform_and_excludes_the_grey_guide():
    with pytest.raises(ValueError):
        layer._options(True, 3, torch.empty(1, 3, 8, 8), None, guide_low=True)
    g = object()
    opt = layer._options(True, 3, torch.empty(1, 3, 8, 8), g, guide_low=True)
    assert (opt.guide_channels, opt.guide_low) == (0, 1)
    with pytest.raises(ValueError):
        layer._options(True, 1, torch.empty(1, 3, 8, 8), g)


def test_sizes_allow_other_guide_channels_only_where_asked():
    p = torch.empty(2, 1, 4, 5)
    ih = torch.empty(2, 3, 16, 20)
    assert layer._sizes(p, ih, grey_ok=True) == (2, 1, 4, 5, 16, 20)
    with pytest.raises(ValueError):
        layer._sizes(p, ih)
    with pytest.raises(ValueError):
        layer._sizes(torch.empty(1, 1, 4, 5), ih, grey_ok=True)


def test_layer_rejects_host_tensors():
    t = torch.zeros(1, 1, 4, 4)
    with pytest.raises(ValueError):
        layer.gf_forward(t, t, torch.zeros(1, 1, 16, 16), 1, 1e-3)


def test_host_step_rejects_device_or_mixed_inputs():
    t = torch.zeros(1, 1, 4, 4)
    with pytest.raises(TypeError):
        layer.gf_step_host(t, t, torch.zeros(1, 1, 16, 16, dtype=torch.float64), torch.zeros(1, 1, 16, 16),
                           1, 1e-3)
