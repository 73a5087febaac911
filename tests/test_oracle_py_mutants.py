"""The pins of the oracle's Python functions are strong enough to catch
plausible mistakes.  The functions are the pinhole camera rays, the
image-gradient regulariser, the shadow map's Gaussian filter, the spotlight
and the painting of picked voxels.

Each case plants one mistake (a dropped term, a wrong sign, factor or index
order) in a copy of `oracle/__init__.py`.  It loads the copy as a module and
runs that function's pins against it: at least one pin must fail.  The
unmodified copy must pass the same pins.  This mirrors the C battery in
`test_oracle_mutants.py`."""
import os
import types

import pytest

import test_oracle_camera as TC
import test_oracle_gradloss as TG

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "__init__.py")

# name -> (pins, text in the oracle, planted mistake)
MUTANTS = {
    "camera_no_half_pixel_x": ("camera", "(2.0 * (px + 0.5) / W - 1.0)", "(2.0 * px / W - 1.0)"),
    "camera_rows_upside_down": ("camera", "(1.0 - 2.0 * (py + 0.5) / H)", "(2.0 * (py + 0.5) / H - 1.0)"),
    "camera_no_aspect": ("camera", "* th * (W / H)", "* th"),
    "camera_tangent_of_full_fov": ("camera", "math.radians(float(cam.fov_y_deg)) / 2.0",
                                   "math.radians(float(cam.fov_y_deg))"),
    "camera_tile_column_major": ("camera", "(ys[:, None] * W + xs[None, :]).ravel()",
                                 "(ys[None, :] * W + xs[:, None]).ravel()"),
    "camera_tiles_width_and_height_swapped": ("camera", "tw, th_ = (8, 4) if tiled is True", "tw, th_ = (4, 8) if tiled is True"),
    "gradloss_first_pixel_sign": ("gradloss", "np.add.at(dE, ra, -2.0 * D)", "np.add.at(dE, ra, 2.0 * D)"),
    "gradloss_no_vertical_pairs": ("gradloss",
                                   "for a, b in ((m[:, :, :-1], m[:, :, 1:]), (m[:, :-1, :], m[:, 1:, :])):",
                                   "for a, b in ((m[:, :, :-1], m[:, :, 1:]),):"),
    "gradloss_error_sign_flipped": ("gradloss", "np.sign(rgb - tgt)", "np.sign(tgt - rgb)"),
    "gradloss_half_gradient": ("gradloss", "np.add.at(dE, rb, 2.0 * D)", "np.add.at(dE, rb, D)"),
    "blur_radius_two_sigma": ("spotlight", "r = int(3.0 * sigma + 0.5)", "r = int(2.0 * sigma + 0.5)"),
    "blur_weights_not_normalised": ("spotlight", "w /= w.sum()", "w /= w.max()"),
    "spot_falloff_inverse_distance": ("spotlight", "fall = lambda P: r_ref * r_ref / np.sum((P - L[:, None]) ** 2, axis=0)",
                                      "fall = lambda P: r_ref / np.sqrt(np.sum((P - L[:, None]) ** 2, axis=0))"),
    "spot_texel_centre_shifted": ("spotlight", "* Wl / 2.0 - 0.5", "* Wl / 2.0"),
    "spot_shadow_not_reversed": ("spotlight", "((1.0 - al) * fall(P))", "(al * fall(P))"),
    "spot_ground_ignores_viewer_alpha": ("spotlight", "out[hit] += (1.0 - A[hit])[:, None] * G", "out[hit] += G"),
    "paint_sum_not_mean": ("paint", "e[hit, :3] = s[hit] / cnt[hit, None]", "e[hit, :3] = s[hit]"),
    "paint_time_not_set": ("paint", "e[hit, 4] = t_d", "e[hit, 4] = 2.0"),
    "paint_counts_unpicked_rays": ("paint", "ok = leaves >= 0", "ok = leaves >= -1"),
}


def _module(src):
    mod = types.ModuleType("oracle_copy")
    mod.__file__ = SRC                           # finds the compiled C part beside the original
    exec(compile(src, SRC, "exec"), mod.__dict__)
    return mod


def _pins(which):
    """The pins of one function, as (name, callable) with fixed parameters."""
    if which == "camera":
        return [("pixel_order_53x37_tiled", lambda: TC.test_pixel_order(53, 37, True)),
                ("pixel_order_33x9_tiled", lambda: TC.test_pixel_order(33, 9, True)),
                ("pinhole_40", lambda: TC.test_directions_follow_the_pinhole(40.0)),
                ("vertical_fov", TC.test_vertical_field_of_view),
                ("generator", TC.test_agrees_with_the_generator),
                ("times_origins", TC.test_times_and_origins)]
    if which == "gradloss":
        return [(n, getattr(TG, n)) for n in dir(TG) if n.startswith("test_")]
    if which == "paint":
        import test_oracle_edit as TE
        return [("paint_means", TE.test_paint_means)]
    import test_oracle_spotlight as TS
    pins = [(n, getattr(TS, n)) for n in dir(TS) if n.startswith("test_") and n != "test_blur_is_the_gaussian_filter"]
    return pins + [("blur_1.5", lambda: TS.test_blur_is_the_gaussian_filter(1.5))]


def _failures(mod, which, monkeypatch):
    import test_oracle_camera
    import test_oracle_gradloss
    import test_oracle_edit
    targets = [test_oracle_camera, test_oracle_gradloss, test_oracle_edit]
    if which == "spotlight":
        import test_oracle_spotlight
        targets.append(test_oracle_spotlight)
    for t in targets:
        monkeypatch.setattr(t, "oracle", mod)
    failed = []
    for name, fn in _pins(which):
        try:
            fn()
        except (AssertionError, ValueError, IndexError, ZeroDivisionError, FloatingPointError):
            failed.append(name)
    return failed


@pytest.mark.parametrize("which", ["camera", "gradloss", "spotlight", "paint"])
def test_unmodified_copy_passes_the_pins(which, monkeypatch):
    if which == "spotlight":
        pytest.importorskip("scipy.ndimage")
    assert _failures(_module(open(SRC).read()), which, monkeypatch) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    which, old, new = MUTANTS[name]
    if which == "spotlight":
        pytest.importorskip("scipy.ndimage")
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    failed = _failures(_module(src.replace(old, new)), which, monkeypatch)
    assert failed, f"no pin caught {name}"
