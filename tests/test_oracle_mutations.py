"""Planted mistakes in the oracle, each caught by a pin.

The pins of test_oracle_pins.py and test_oracle_cnn.py tie the oracle to the
paper and to the mathematics.  They are only worth something if a plausible
mistake in the oracle (a dropped term, a wrong sign, factor or index, a
transposed operand, a miscount) makes one of them fail.  Each test here plants
one such mistake in an oracle function, for the duration of the test only
(pytest's monkeypatch, on the CPU), runs the pin that should catch it and
requires that pin to fail.  Nothing here touches the CUDA library.
"""
import inspect
import textwrap

import numpy as np
import pytest

import test_oracle_cnn as cnn_pins
import test_oracle_pins as pins
from oracle import basis, cnn, fem, krylov
from oracle import multigrid as mg


def must_fail(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def mutant(owner, name, *edits):
    """The oracle function owner.name (owner a module or a class) with each
    (old, new) of `edits` made in its source (every `old` found exactly once),
    compiled in a copy of the namespace of the module that defines it."""
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    ns = dict(fn.__globals__)
    exec(compile(src, f"<planted {owner.__name__}.{name}>", "exec"), ns)
    return ns[name]


def plant(monkeypatch, module, name, old, new):
    monkeypatch.setattr(module, name, mutant(module, name, (old, new)))


# --- the operator: eq. (ipbrinkman), eq. (Brinkman-weak) ---------------------------

def test_half_penalty(monkeypatch):
    """sigma_j = (k+1)(k+2)/h_j (Sec. 4.1) with a factor 1/2 lost (or the 2 of
    2 mu sigma dropped): consistency survives, the hand-derived energies do not."""
    orig = fem.penalty
    monkeypatch.setattr(fem, "penalty", lambda k, h: 0.5 * orig(k, h))
    must_fail(pins.test_energy_closed_forms, 1.0, 0.0)


def test_interior_consistency_sign(monkeypatch):
    """The consistency terms -mu <{du/dn}, [v]> - mu <{dv/dn}, [u]> on interior
    faces with the wrong sign: the penalty part of a face matrix is linear in
    sigma, so F(sigma) - 2 F(0) flips exactly the consistency part."""
    orig = fem.face_matrices
    monkeypatch.setattr(fem, "face_matrices",
                        lambda S, mu, sigma, e: orig(S, mu, sigma, e) - 2.0 * orig(S, mu, 0.0, e))
    must_fail(pins.test_polynomial_reproduction, 2, 1, 4, 1.0)


def test_boundary_consistency_sign(monkeypatch):
    orig = fem.boundary_face_matrix
    monkeypatch.setattr(fem, "boundary_face_matrix",
                        lambda S, mu, sigma, e, high: orig(S, mu, sigma, e, high) - 2.0 * orig(S, mu, 0.0, e, high))
    must_fail(pins.test_polynomial_reproduction, 2, 1, 4, 1.0)


def test_boundary_face_on_the_wrong_side(monkeypatch):
    """The Nitsche terms of a boundary cell taken on its opposite face (outward
    normal mixed up)."""
    orig = fem.boundary_face_matrix
    monkeypatch.setattr(fem, "boundary_face_matrix",
                        lambda S, mu, sigma, e, high: orig(S, mu, sigma, e, not high))
    must_fail(pins.test_polynomial_reproduction, 2, 1, 4, 1.0)


def _cell_matrices_with(monkeypatch, change):
    orig = fem.cell_matrices
    monkeypatch.setattr(fem, "cell_matrices", lambda S: change(*orig(S)))


def test_divergence_sign(monkeypatch):
    """-(q, div u) with the sign flipped: the pressure of the solution flips."""
    _cell_matrices_with(monkeypatch, lambda K, M, B: (K, M, -B))
    must_fail(pins.test_literal_channel_rhs_closed_form, 1)


def test_mass_term_dropped(monkeypatch):
    _cell_matrices_with(monkeypatch, lambda K, M, B: (K, 0.0 * M, B))
    must_fail(pins.test_energy_closed_forms, 0.0, 1.0)


def test_viscous_volume_term_dropped(monkeypatch):
    _cell_matrices_with(monkeypatch, lambda K, M, B: (0.0 * K, M, B))
    must_fail(pins.test_energy_closed_forms, 1.0, 0.0)


def test_quadrature_one_point_short(monkeypatch):
    """k+1 instead of k+2 Gauss points per direction: the mass matrix of the
    velocity space is no longer integrated exactly."""
    orig = fem._tensor_quad
    monkeypatch.setattr(fem, "_tensor_quad", lambda d, npts: orig(d, npts - 1))
    must_fail(pins.test_energy_closed_forms, 0.0, 1.0)


def test_gauss_weights_on_the_wrong_interval(monkeypatch):
    """Gauss weights of [-1, 1] (summing to 2) used on the unit interval."""
    orig = basis.gauss
    monkeypatch.setattr(basis, "gauss", lambda npts: (orig(npts)[0], 2.0 * orig(npts)[1]))
    must_fail(pins.test_energy_closed_forms, 0.37, 2.5)


def test_nitsche_boundary_data_sign(monkeypatch):
    """The boundary-data term -mu <dv/dn, g> of F (eq. BCh) with the wrong sign."""
    plant(monkeypatch, fem, "load_vector", "- mu * nu * D[a]", "+ mu * nu * D[a]")
    must_fail(pins.test_polynomial_reproduction, 2, 1, 4, 1.0)


def test_normal_velocity_constrained_on_one_side_only(monkeypatch):
    """The strongly imposed normal velocity (reading of eq. BCh) set on the
    x_i = 0 faces only, the x_i = 1 faces left free."""
    monkeypatch.setattr(fem.Space, "constrained", mutant(
        fem.Space, "constrained", ("on = (idx[:, i] == 0) | (idx[:, i] == self.N)", "on = idx[:, i] == 0")))
    must_fail(pins.test_literal_channel_rhs_closed_form, 1)


def test_evaluated_divergence_missing_the_mesh_size(monkeypatch):
    """Point evaluation of div u without the 1/h of the reference derivative."""
    plant(monkeypatch, fem, "evaluate", "div[q] += coef[a] * grads[a, 0, kd] / h",
          "div[q] += coef[a] * grads[a, 0, kd]")
    must_fail(pins.test_load_vector_divergence_source, 2, 1, 3)


def test_pressure_weights_missing_cell_measure(monkeypatch):
    """w_i = (1, q_i) without the h^d of the cell: the pressure rows built from
    them no longer integrate the source."""
    monkeypatch.setattr(fem.Space, "pressure_weights", mutant(
        fem.Space, "pressure_weights", ("np.ones(idx.shape[0]) * self.h ** self.d", "np.ones(idx.shape[0])")))
    must_fail(pins.test_divergence_is_exact_pointwise, 2, 1, 3)


# --- right-hand side: eq. (BCh), the divergence source ----------------------------

def _load_vector_with(monkeypatch, change):
    orig = fem.load_vector

    def planted(S, *args, **kw):
        b = orig(S, *args, **kw)
        if kw.get("div_source") is not None:
            b[S.n_u:] = change(b[S.n_u:], S)
        return b
    monkeypatch.setattr(fem, "load_vector", planted)


def test_divergence_source_sign(monkeypatch):
    _load_vector_with(monkeypatch, lambda bp, S: -bp)
    must_fail(pins.test_load_vector_divergence_source, 2, 1, 3)


def test_divergence_source_missing_cell_measure(monkeypatch):
    _load_vector_with(monkeypatch, lambda bp, S: bp / S.h ** S.d)
    must_fail(pins.test_load_vector_divergence_source, 2, 1, 3)


# --- transfers and coarse levels: Sec. 3.1, Sec. 4.1 -------------------------------

def test_prolongation_pressure_block_scaled(monkeypatch):
    """Pressure injection with a stray factor (an averaging weight 1/2 taken
    over from the restriction)."""
    import scipy.sparse as sp
    orig = mg.prolongation

    def planted(Sc, Sf):
        scale = np.ones(Sf.ndof)
        scale[Sf.n_u:] = 0.5
        return (sp.diags(scale) @ orig(Sc, Sf)).tocsr()
    monkeypatch.setattr(mg, "prolongation", planted)
    must_fail(pins.test_prolongation_reproduces_coarse_functions, 2, 1, 2)


def test_coarse_coefficient_averaged_the_other_way(monkeypatch):
    orig = mg.coarsen_c
    monkeypatch.setattr(mg, "coarsen_c",
                        lambda c, d, mode="arithmetic": orig(c, d, "harmonic" if mode == "arithmetic" else "arithmetic"))
    must_fail(pins.test_coarsen_is_arithmetic_mean_of_the_coefficient)


# --- smoother, patches and V-cycle: Sec. 3.2, Sec. 3.3 -------------------------------

def test_patches_coloured_mod_two(monkeypatch):
    """2^d colours (v_e mod 2) instead of 3^d: patches of one colour then share
    dofs and couple."""
    orig = mg.patches

    def planted(S):
        cols = orig(S)
        verts = np.concatenate([v for v, _ in cols])
        dofs = np.concatenate([p for _, p in cols])
        key = sum((verts[:, e] % 2) * 2 ** e for e in range(S.d))
        return [(verts[key == c], dofs[key == c]) for c in range(2 ** S.d)]
    monkeypatch.setattr(mg, "patches", planted)
    must_fail(pins.test_patch_count_and_colours, 2, 1)


@pytest.mark.parametrize("count", [lambda H, j, m: m * 2 ** j,
                                   lambda H, j, m: m * 2 ** (H.J - j + 1),
                                   lambda H, j, m: m * (H.J - j + 1)],
                         ids=["2^j", "2^(J-j+1)", "linear"])
def test_variable_cycle_miscounts(monkeypatch, count):
    """m(j) = m(J) 2^(J-j) (Sec. 3.2) replaced by plausible miscounts."""
    monkeypatch.setattr(mg, "smoothing_steps",
                        lambda H, j, m_fine, variable: count(H, j, m_fine) if variable else m_fine)
    must_fail(pins.test_variable_cycle_smoothing_counts_against_dense_construction, *pins.SMOOTHING_COUNT_CASES[2])


def test_patch_mean_constraint_on_every_dof(monkeypatch):
    """The bordering row of the patch problem (zero pressure mean, Sec. 3.3)
    taken over all patch dofs, velocities included.  On a one-patch mesh this
    only moves the pressure constant; with several patches the multiplier of
    the constraint then enters the velocity rows, which the two-grid built
    from explicit Ritz projections sees."""
    plant(monkeypatch, mg, "patch_inverses", "wv = w[dofs]", "wv = np.ones(dofs.shape)")
    must_fail(pins.test_two_grid_against_dense_ritz_construction, 2, 1)


def test_colour_updates_deferred_to_the_end_of_the_sweep(monkeypatch):
    """Every colour's corrections computed from the residual at the start of
    the sweep (the colours no longer multiplicative)."""
    monkeypatch.setattr(mg, "smooth_step", mutant(
        mg, "smooth_step",
        ("    x = x.copy()\n    for col in order:", "    x = x.copy()\n    pend = []\n    for col in order:"),
        ("        for dofs, delta in upd:\n            x[dofs] += delta\n    return x",
         "        pend.extend(upd)\n    for dofs, delta in pend:\n        x[dofs] += delta\n    return x")))
    must_fail(pins.test_colour_pass_equals_patch_by_patch, 2, 1)


def test_post_smoothing_dropped(monkeypatch):
    """The V-cycle without its post-smoothing steps: no longer symmetric."""
    plant(monkeypatch, mg, "vcycle_level",
          "    x = x + H.P[j] @ xc\n    for _ in range(m):\n        x = smooth(x)\n    return x",
          "    x = x + H.P[j] @ xc\n    return x")
    must_fail(pins.test_vcycle_is_symmetric, 2, 1, 3, False)


def test_boundary_patches_keep_pressure_only_corners(monkeypatch):
    """Boundary-vertex patches (Sec. 3.3) without the rule that drops a patch
    holding no velocity dof (an RT_0 corner: one pressure, zero under the
    mean-zero constraint)."""
    plant(monkeypatch, mg, "boundary_patches_of",
          "        if not np.any(dofs < S.n_u):\n            continue\n", "")
    must_fail(pins.test_boundary_patch_sizes_by_hand, 2, 0, 4, {3: 12})


def test_boundary_patch_vertex_off_by_one(monkeypatch):
    """The vertex of a boundary dof's patch one cell off along every direction."""
    plant(monkeypatch, mg, "boundary_patches_of", "v = hi[cand, e] + choice[e]", "v = hi[cand, e] + choice[e] + 1")
    must_fail(pins.test_boundary_patch_sizes_by_hand, 2, 1, 4, {8: 4, 18: 12})


def test_additive_damping_ignored(monkeypatch):
    """The additive variant (not the paper's smoother) without its damping omega."""
    plant(monkeypatch, mg, "additive_step", "return x + omega * d", "return x + d")
    must_fail(pins.test_additive_step_is_sum_of_ritz_corrections, 2, 1)


def test_forward_sweep_only(monkeypatch):
    """The smoothing step without its backward sweep (colours 0..C-1 only):
    the V-cycle is no longer symmetric."""
    def planted(L, x, b):
        x = x.copy()
        for col in range(len(L.colours)):
            upd = []
            for dofs, Sv, Arows in L.colour_groups(col):
                r = (b[dofs.ravel()] - Arows @ x).reshape(dofs.shape)
                upd.append((dofs, np.einsum("pij,pj->pi", Sv, r)))
            for dofs, delta in upd:
                x[dofs] += delta
        return x
    monkeypatch.setattr(mg, "smooth_step", planted)
    must_fail(pins.test_vcycle_is_symmetric, 2, 1, 3, False)


def test_coarse_solve_bordered_with_ones(monkeypatch):
    """The coarsest solve (B_0 = A_0^{-1} on the mean-zero space, Sec. 3.2)
    bordered with ones over every free dof instead of the pressure weights."""
    monkeypatch.setattr(mg.Hierarchy, "__init__", mutant(
        mg.Hierarchy, "__init__", ("Bm[:nf, nf] = wf", "Bm[:nf, nf] = 1.0"), ("Bm[nf, :nf] = wf", "Bm[nf, :nf] = 1.0")))
    must_fail(pins.test_two_grid_against_dense_ritz_construction, 2, 1)


def test_residual_not_updated_before_restriction(monkeypatch):
    """The coarse level given the restricted right-hand side b instead of the
    residual b - A x after pre-smoothing (the garbled coarse-correction line
    of Sec. 3.2 read without its A x): the V-cycle with that one line changed,
    against the dense two-grid built from the paper's construction."""
    def planted(H, j, b, m_fine, variable, additive=0.0):
        if j == 0:
            return mg.coarse_solve(H, b)
        L = H.levels[j]
        m = mg.smoothing_steps(H, j, m_fine, variable)
        x = np.zeros_like(b)
        for _ in range(m):
            x = mg.smooth_step(L, x, b)
        r = b.copy()                      # planted: A x not subtracted
        r[L.cm] = 0.0
        bc = H.P[j].T @ r
        bc[H.levels[j - 1].cm] = 0.0
        x = x + H.P[j] @ planted(H, j - 1, bc, m_fine, variable)
        for _ in range(m):
            x = mg.smooth_step(L, x, b)
        return x
    monkeypatch.setattr(mg, "vcycle_level", planted)
    must_fail(pins.test_two_grid_against_dense_ritz_construction, 2, 1)


# --- the outer flexible GMRES (Sec. 3.2, Sec. 4.1) -----------------------------------

def test_fgmres_update_with_the_unpreconditioned_basis(monkeypatch):
    plant(monkeypatch, krylov, "fgmres", "x = x + Z[:kdone].T @ y", "x = x + V[:kdone].T @ y")
    must_fail(pins.test_fgmres_matches_dense_solve)


def test_fgmres_givens_sine_sign(monkeypatch):
    plant(monkeypatch, krylov, "fgmres", "sn[i] = Hm[i + 1, i] / den", "sn[i] = -Hm[i + 1, i] / den")
    must_fail(pins.test_fgmres_residual_is_the_krylov_minimum)


def test_fgmres_gram_schmidt_index(monkeypatch):
    plant(monkeypatch, krylov, "fgmres", "Hm[l, i] = np.dot(w, V[l])", "Hm[l, i] = np.dot(w, V[i])")
    must_fail(pins.test_fgmres_residual_is_the_krylov_minimum)


# --- the learned guess's network (oracle/cnn.py) -----------------------------------

def test_convolution_taps_flipped(monkeypatch):
    """True convolution (kernel flipped) instead of the correlation the network uses."""
    orig = cnn.conv3x3
    monkeypatch.setattr(cnn, "conv3x3", lambda x, w, b: orig(x, w[:, :, ::-1, ::-1], b))
    must_fail(cnn_pins.test_conv_matches_direct_loops)


def test_input_gradient_dropped(monkeypatch):
    orig = cnn.conv3x3_backward

    def planted(x, w, gy):
        gx, gw, gb = orig(x, w, gy)
        return np.zeros_like(gx), gw, gb
    monkeypatch.setattr(cnn, "conv3x3_backward", planted)
    must_fail(cnn_pins.test_backward_matches_finite_differences)


def test_weight_gradient_taps_flipped(monkeypatch):
    orig = cnn.conv3x3_backward

    def planted(x, w, gy):
        gx, gw, gb = orig(x, w, gy)
        return gx, gw[:, :, ::-1, ::-1].copy(), gb
    monkeypatch.setattr(cnn, "conv3x3_backward", planted)
    must_fail(cnn_pins.test_backward_matches_finite_differences)


def test_relu_derivative_dropped(monkeypatch):
    plant(monkeypatch, cnn, "loss_and_grads", "g = g * (pre[li] > 0.0)", "g = g")
    must_fail(cnn_pins.test_backward_matches_finite_differences)
