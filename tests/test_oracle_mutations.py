"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in one oracle routine, on the CPU: a
dropped term, a wrong sign, index or axis, a transposed operand, a wrong
constant or an off-by-one.  It does so by editing the routine's source text and
re-compiling it in the oracle's namespace.  The case then requires a named pin
(a test in tests/test_oracle_*.py) to fail on the mutant with an
AssertionError.  A case that stayed green would mean that the pins cannot tell
that mistake from the method, so every case here names the pin that catches it.
"""
import inspect
import textwrap

import pytest

from oracle import toi_oracle as O

import test_oracle_3d as T3
import test_oracle_adjoint as TA
import test_oracle_imaging as TI
import test_oracle_localise as TL
import test_oracle_trigger as TT


def _mutant(name, old, new):
    """The oracle routine `name` with the one occurrence of `old` in its source
    replaced by `new`, compiled against the oracle module's globals."""
    src = textwrap.dedent(inspect.getsource(getattr(O, name)))
    assert src.count(old) == 1, f"{name}: mutation site {old!r} not found exactly once"
    ns = {}
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), vars(O), ns)
    return ns[name]


def _row(name):
    return next(r for r in T3._table2() if r[0] == name)


# (id, routine, original text, mutated text, the pin that must fail)
CASES = [
    # ---- S1: selection, weights, plane fit (Sections 3, 3.1, 3.3, 3.5)
    ("weights dropped from the hand average", "sample_weights_and_values",
     "c_q = wp[:, :, pa] * v[:, :, pa] + wp[:, :, pb] * v[:, :, pb]",
     "c_q = w_q * 0.5 * (v[:, :, pa] + v[:, :, pb])",
     TI.test_sample_weights_pol_average_by_hand),
    ("flags ignored", "sample_weights_and_values",
     "wp = np.where(f, 0.0, np.asarray(weight, dtype=np.float64))",
     "wp = np.asarray(weight, dtype=np.float64)",
     TI.test_sample_weights_pol_average_by_hand),
    ("zero-weight samples kept in the plane fit", "prepare",
     "sel = w_q > 0", "sel = w_q >= 0",
     TI.test_flagged_samples_do_not_move_the_plane),
    ("wavelength scaling inverted", "wavelength_baselines",
     "k = np.asarray(freq_hz, dtype=np.float64) / C_LIGHT",
     "k = C_LIGHT / np.asarray(freq_hz, dtype=np.float64)",
     TI.test_point_source_off_centre_closed_form),
    ("cloud not centred", "svd_basis",
     "Bt = B_sel - B_sel.mean(axis=0, keepdims=True)", "Bt = B_sel.copy()",
     TI.test_svd_planted_plane_normal),
    ("largest instead of smallest singular vector", "svd_basis",
     "v3 = Vt[2].copy()", "v3 = Vt[0].copy()",
     TI.test_svd_planted_plane_normal),
    ("left-handed basis", "svd_basis",
     "v2 = np.cross(v3, v1)", "v2 = np.cross(v1, v3)",
     TI.test_svd_planted_plane_normal),
    ("sign in the area Jacobian", "omega_of",
     "V[0, 0] * V[1, 1] - V[1, 0] * V[0, 1]", "V[0, 0] * V[1, 1] + V[1, 0] * V[0, 1]",
     TI.test_omega_is_the_cofactor_for_any_rotation),
    ("xi and eta swapped", "tilt_of",
     "return V[2, 0] / V[2, 2], V[2, 1] / V[2, 2]", "return V[2, 1] / V[2, 2], V[2, 0] / V[2, 2]",
     TI.test_svd_planted_plane_normal),
    # ---- S2/S3: coordinates and gridding (Section 3.2, Section 4.1 stage 3)
    ("kernel argument not scaled by 2/W", "es_kernel",
     "z = 2.0 * np.asarray(x, dtype=np.float64) / W", "z = np.asarray(x, dtype=np.float64) / W",
     TI.test_es_kernel_values),
    ("kernel not normalised to psi(0) = 1", "es_kernel",
     "np.sqrt(1.0 - zz * zz) - 1.0", "np.sqrt(1.0 - zz * zz)",
     TI.test_es_kernel_values),
    ("sign of the column coordinate", "grid_coords",
     "g1 = G / 2 - np.asarray(r1) * beta * G", "g1 = G / 2 + np.asarray(r1) * beta * G",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("row coordinate scaled by N instead of G", "grid_coords",
     "g2 = G / 2 + np.asarray(r2) * beta * G", "g2 = G / 2 + np.asarray(r2) * beta * N",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("first tap by floor instead of ceil", "tap_start",
     "np.ceil(g - W / 2.0)", "np.floor(g - W / 2.0)",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("row kernel evaluated at the column coordinate", "grid_es",
     "wy = [es_kernel(k2 + b - g2, W, beta) for b in range(W)]",
     "wy = [es_kernel(k2 + b - g1, W, beta) for b in range(W)]",
     TI.test_gridding_degridding_adjoint),
    ("grid transposed", "grid_es",
     "idx = (k2 + b) * G + (k1 + a)", "idx = (k1 + a) * G + (k2 + b)",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("degridding conjugates the grid", "degrid_es",
     "out += grid[k2 + b, k1 + a] * (wx * wy)", "out += np.conj(grid[k2 + b, k1 + a]) * (wx * wy)",
     TI.test_gridding_degridding_adjoint),
    # ---- S4/S5: inverse FFT, correction, normalisation (Section 3.2, Eq. 11)
    ("forward instead of inverse transform", "ifft_centred",
     'np.fft.ifft2(np.fft.ifftshift(grid), norm="forward")',
     'np.fft.fft2(np.fft.ifftshift(grid), norm="backward")',
     TI.test_gridded_image_matches_bruteforce_dft),
    ("transform not centred", "ifft_centred",
     'np.fft.ifft2(np.fft.ifftshift(grid), norm="forward")',
     'np.fft.ifft2(grid, norm="forward")',
     TI.test_gridded_image_matches_bruteforce_dft),
    ("Fourier integral at half the frequency", "es_fourier",
     "np.cos(2 * np.pi * np.outer(f, x))", "np.cos(np.pi * np.outer(f, x))",
     TI.test_es_fourier_quadrature_vs_adaptive),
    ("correction sampled at j / N instead of j / G", "correction_vector",
     "return es_fourier(j / G, W, beta)", "return es_fourier(j / N, W, beta)",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("omega dropped from the normalisation", "tilted_image",
     "return img / (ph[:, None] * ph[None, :]) / (omega * sumw)",
     "return img / (ph[:, None] * ph[None, :]) / sumw",
     TI.test_point_source_at_phase_centre),
    ("correction on one axis only", "tilted_image",
     "return img / (ph[:, None] * ph[None, :]) / (omega * sumw)",
     "return img / ph[None, :] / (omega * sumw)",
     TI.test_gridded_image_matches_bruteforce_dft),
    ("Hermitian half without the conjugate", "hermitian_half",
     "S = 0.5 * (grid + np.conj(grid[idx][:, idx]))", "S = 0.5 * (grid + grid[idx][:, idx])",
     TI.test_hermitian_half_gives_real_image),
    ("brute-force image with the column axis mirrored", "dirty_image_dft",
     "t1 = -beta * (cols - N // 2)", "t1 = beta * (cols - N // 2)",
     TI.test_gridded_image_matches_bruteforce_dft),
    # ---- S6: re-projection (Section 3.3, Appendix A)
    ("sign of the eta term", "reproject_map_reduced",
     "yp = y + r0 * z * eta", "yp = y - r0 * z * eta",
     TI.test_reprojection_reduced_equals_wcs),
    ("small-angle form of z", "reproject_map_reduced",
     "z = q / (1.0 + np.sqrt(1.0 - q))", "z = q / 2.0",
     TI.test_reprojection_reduced_equals_wcs),
    ("sign of the xi term on the WCS route", "reproject_map_wcs",
     "xs = np.cos(theta) * np.sin(phi) + xi * (1 - np.sin(theta))",
     "xs = np.cos(theta) * np.sin(phi) - xi * (1 - np.sin(theta))",
     TI.test_reprojection_reduced_equals_wcs),
    ("fixed-point step with the wrong sign", "reproject_source_at",
     "p1 = p1o - (m1 - p1)", "p1 = p1o + (m1 - p1)",
     TI.test_reprojection_gather_inverts_map),
    ("cell converted from arcminutes instead of arcseconds", "reproject",
     "cell_arcsec / 3600.0", "cell_arcsec / 60.0",
     TI.test_reproject_moves_a_point_where_the_wcs_route_maps_it),
    ("interpolation weights of the two axes swapped", "bilinear",
     "v = ((1 - fb) * ((1 - fa) * pad[b0c, a0c] + fa * pad[b0c, a0c + 1]) +",
     "v = ((1 - fa) * ((1 - fb) * pad[b0c, a0c] + fb * pad[b0c, a0c + 1]) +",
     TI.test_bilinear_exact_on_planes),
    # ---- reverse mode (Section 1's adjoint route)
    ("bilinear transpose spreads to the wrong neighbour", "bilinear_adjoint",
     "np.add.at(out, (b0, a0 + 1), (1 - fb) * fa * g)",
     "np.add.at(out, (b0 + 1, a0), (1 - fb) * fa * g)",
     TA.test_bilinear_adjoint_is_the_transpose),
    ("adjoint transform with the inverse's sign", "tilted_image_adjoint",
     "return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(pad)))",
     'return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(pad), norm="forward"))',
     TA.test_tilted_adjoint_matches_dft_adjoint),
    ("correction dropped from the adjoint", "tilted_image_adjoint",
     "U = grad_tilted / (ph[:, None] * ph[None, :]) / (omega * sumw)",
     "U = grad_tilted / (omega * sumw)",
     lambda: TA.test_image_adjoint_identity(1, False)),
    ("1 / sum w term dropped from the weight gradient", "image_snapshot_adjoint",
     "gw = (np.conj(g) * vis[:, :, p].astype(np.complex128)).real - dot / r[\"sumw\"]",
     "gw = (np.conj(g) * vis[:, :, p].astype(np.complex128)).real",
     TA.test_weight_gradient_matches_finite_differences),
    ("visibility gradient without the hand's weight", "image_snapshot_adjoint",
     "grad_vis[:, :, p] = np.where(sel, wp[:, :, p] * g, 0.0)",
     "grad_vis[:, :, p] = np.where(sel, g, 0.0)",
     lambda: TA.test_image_adjoint_identity(4, True)),
    ("w term dropped from d/dl", "point_source_gradient",
     "dl = -2j * np.pi * k[None, :] * (uvw[:, 0:1] - uvw[:, 2:3] * l / n) * flux * v",
     "dl = -2j * np.pi * k[None, :] * uvw[:, 0:1] * flux * v",
     TA.test_point_source_gradient_matches_finite_differences),
    ("w term dropped from the point-source phase", "point_source_vis",
     " + uvw[:, 2:3] * (n - 1.0)) * k[None, :]", ") * k[None, :]",
     TA.test_point_source_gradient_matches_finite_differences),
    # ---- localisation windows
    ("point-source phase with the wrong sign", "point_source_vis",
     "v = flux * np.exp(-2j * np.pi * ph)", "v = flux * np.exp(2j * np.pi * ph)",
     TL.test_coplanar_peak_is_flux_over_omega_at_the_named_pixel),
    ("window rows and columns swapped", "window_axes",
     "return np.arange(j2c, j2c + size), np.arange(j1c, j1c + size)",
     "return np.arange(j1c, j1c + size), np.arange(j2c, j2c + size)",
     TL.test_coplanar_peak_is_flux_over_omega_at_the_named_pixel),
    ("window adjoint without the conjugate phase", "window_adjoint_exact",
     "e1 = np.exp(-2j * np.pi * np.outer(p[\"r\"][:, 0], t1))",
     "e1 = np.exp(2j * np.pi * np.outer(p[\"r\"][:, 0], t1))",
     TL.test_window_adjoint_is_the_transpose),
    ("source direction through V instead of V^T", "source_of_pixel",
     "s = V.T @ tau + np.array([0.0, 0.0, 1.0])", "s = V @ tau + np.array([0.0, 0.0, 1.0])",
     TL.test_coplanar_peak_is_flux_over_omega_at_the_named_pixel),
    ("sign of the residual cotangent", "localise",
     "gM = -2.0 * R", "gM = 2.0 * R",
     TL.test_source_gradient_matches_finite_differences),
    ("data term dropped from the weight gradient", "localise",
     "(np.conj(gq_d) * vis[:, :, p].astype(np.complex128)).real - dot", "- dot",
     TL.test_weight_gradient_matches_finite_differences),
    # ---- near-coplanar mode (Section 3.4, Appendix B, Table 2)
    ("transposed index of V in t3", "t3_of",
     "2.0 * t2 * V[1, 2]", "2.0 * t2 * V[2, 1]",
     T3.test_t3_lies_on_the_sphere_and_matches_the_printed_root),
    ("Jacobi-Anger coefficients with (-i)^k", "chebyshev_coeffs",
     "c = 2.0 * (1j ** k) * J", "c = 2.0 * ((-1j) ** k) * J",
     T3.test_jacobi_anger_series),
    ("Chebyshev recurrence with the wrong sign", "chebyshev_T",
     "T[..., k] = 2.0 * s * T[..., k - 1] - T[..., k - 2]",
     "T[..., k] = 2.0 * s * T[..., k - 1] + T[..., k - 2]",
     T3.test_jacobi_anger_series),
    ("Phi_max over the full r3 range", "slab_plan",
     "phi = 2.0 * math.pi * t3max * (r3max - r3min) / 2.0",
     "phi = 2.0 * math.pi * t3max * (r3max - r3min)",
     lambda: T3.test_table2_rows(_row("MeerKAT"))),
    ("alpha_slab without the factor 2", "slab_plan",
     "alpha_slab = 2.0 * math.pi * t3max * dr3", "alpha_slab = math.pi * t3max * dr3",
     lambda: T3.test_table2_rows(_row("MeerKAT"))),
    ("slab offset over the full width", "slab_of",
     "s = (r3 - plan[\"centres\"][p]) / plan[\"dr3\"]",
     "s = (r3 - plan[\"centres\"][p]) / (2.0 * plan[\"dr3\"])",
     T3.test_slab_assignment),
    ("slab phase with the wrong sign", "tilted_image_3d",
     "slab_phase = np.exp(2j * math.pi * plan[\"centres\"][p] * T3)",
     "slab_phase = np.exp(-2j * math.pi * plan[\"centres\"][p] * T3)",
     T3.test_moment_image_matches_the_exact_3d_dft),
    ("r3 t3 term dropped from the exact 3-D image", "dirty_image_3d_dft",
     " + np.outer(tt3, r[:, 2]))", ")",
     T3.test_moment_image_matches_the_exact_3d_dft),
    # ---- S7 tLISI (the stand-in definition) and S8 candidates
    ("second difference taken against I0", "tlisi",
     "b = np.asarray(I2, np.float64) - np.asarray(I1, np.float64)",
     "b = np.asarray(I2, np.float64) - np.asarray(I0, np.float64)",
     TT.test_tlisi_identical_differences_is_one),
    ("C2 = 0.03 L^2 instead of (0.03 L)^2", "tlisi",
     "C2 = (0.03 * L) ** 2", "C2 = 0.03 * L ** 2",
     TT.test_tlisi_hand_example_2x2_tiles),
    ("mean not removed from the variance", "tlisi",
     "va = (at * at).sum(-1) / n - mu_a * mu_a", "va = (at * at).sum(-1) / n",
     TT.test_tlisi_hand_example_2x2_tiles),
    ("dynamic range without the absolute value", "tlisi",
     "L = max(np.abs(I0).max(), np.abs(I1).max(), np.abs(I2).max())",
     "L = max(I0.max(), I1.max(), I2.max())",
     TT.test_tlisi_hand_example_2x2_tiles),
    ("twiddle of the second quadrant", "twiddle",
     "return -s, c", "return s, c",
     TT.test_twiddles_match_libm),
    ("twiddle angle a quarter too small", "twiddle",
     "r = (PI_2 * float(a)) / float(S)", "r = (PI_2 * float(a)) / float(4 * S)",
     TT.test_twiddles_match_libm),
    ("harmonic sum normalised by h instead of sqrt(h)", "periodic_scores",
     "best = np.maximum(best, H / roots[h])", "best = np.maximum(best, H / float(h))",
     TT.test_periodogram_matches_fft),
    ("last harmonic dropped", "periodic_scores",
     "if i * f > F:", "if i * f >= F:",
     TT.test_periodic_score_at_the_highest_frequency),
    ("non-periodic score sums tLISI instead of 1 - tLISI", "nonperiodic_scores",
     "acc = acc + (1.0 - x[t])", "acc = acc + x[t]",
     TT.test_nonperiodic_dip_found),
    ("sample instead of population deviation", "threshold",
     "var = pairwise_sum(d * d) / float(n)", "var = pairwise_sum(d * d) / float(n - 1)",
     TT.test_threshold_by_hand),
    ("pairwise split rounded up", "pairwise_sum",
     "mid = lo + n // 2", "mid = lo + (n + 1) // 2",
     TT.test_pairwise_sum_tree),
    ("4-connected instead of 8-connected tiles", "connected_boxes",
     "if 0 <= ny < nty and 0 <= nx < ntx and mask[ny, nx] and lab[ny, nx] < 0:",
     "if abs(dy) + abs(dx) == 1 and 0 <= ny < nty and 0 <= nx < ntx and mask[ny, nx] "
     "and lab[ny, nx] < 0:",
     TT.test_connected_boxes_by_hand),
    ("box end not half-open", "connected_boxes",
     "(max(xs) + 1) * T", "max(xs) * T",
     TT.test_connected_boxes_by_hand),
    ("4 sigma for the periodic search", "candidates",
     "k = 5.0", "k = 4.0",
     TT.test_periodic_planted_tile_found),
    ("candidates at the threshold itself", "candidates",
     "mask = (sc > thr)", "mask = (sc >= thr)",
     TT.test_threshold_strict_and_flat),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")    # a mutant may produce NaN
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(case, monkeypatch):
    _, name, old, new, pin = case
    pin()                                   # green on the oracle as it stands
    monkeypatch.setattr(O, name, _mutant(name, old, new))
    with pytest.raises(AssertionError):
        pin()
