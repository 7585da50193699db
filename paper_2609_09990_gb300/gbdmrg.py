"""Python binding of libgbdmrg (include/gbdmrg.h, include/gbdmrg_test.h).

Argument marshalling only: every step of the sweep runs inside the C/CUDA
library.  The names mirror the C entry points.  If the shared library has not
been built, loading raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbdmrg.so")

GBD_OK = 0
GBD_ERR_ARG, GBD_ERR_OOM, GBD_ERR_CUDA, GBD_ERR_NOCONV, GBD_ERR_TIMEOUT, GBD_ERR_STATE = -1, -2, -3, -4, -5, -6
GBD_FP64, GBD_TF32, GBD_BF16 = 0, 1, 2
GBD_PRECOND_DIAG, GBD_PRECOND_LEARNED, GBD_PRECOND_OLSEN, GBD_PRECOND_PCG = 0, 1, 2, 3
ERRORS = {-1: "GBD_ERR_ARG", -2: "GBD_ERR_OOM", -3: "GBD_ERR_CUDA", -4: "GBD_ERR_NOCONV",
          -5: "GBD_ERR_TIMEOUT", -6: "GBD_ERR_STATE"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class gbd_problem(C.Structure):
    _fields_ = [("n_orb", C.c_int32), ("n_elec", C.c_int32), ("two_sz", C.c_int32), ("n_chol", C.c_int32),
                ("h", _dp), ("chol", _dp), ("e_core", C.c_double)]


class gbd_schedule(C.Structure):
    _fields_ = [("n_sweeps", C.c_int32), ("bond_dim", _ip), ("davidson_tol", _dp),
                ("davidson_max_iter", C.c_int32), ("davidson_max_subspace", C.c_int32),
                ("precision", C.c_int32), ("preconditioner", C.c_int32), ("seed", C.c_uint64),
                ("svd_cutoff", C.c_double), ("fp64_refine", C.c_int32)]


class gbd_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("sweep_energies", _dp), ("rdm1", _dp), ("rdm2", _dp),
                ("max_discarded_weight", C.c_double), ("n_matvec", C.c_int64), ("status", C.c_int32)]


class gbd_stats(C.Structure):
    _fields_ = [("sigma_flops", C.c_double), ("sigma_ms", C.c_double), ("env_flops", C.c_double),
                ("env_ms", C.c_double), ("enlarge_ms", C.c_double), ("davidson_ms", C.c_double),
                ("truncate_ms", C.c_double), ("step_ms", C.c_double), ("n_sigma", C.c_int64),
                ("n_steps", C.c_int64), ("kernel_launches", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("max_discarded_weight", C.c_double),
                ("sigma_flops_exec", C.c_double), ("tc_ms", C.c_double), ("tc_flops", C.c_double),
                ("n_sigma_tc", C.c_int64), ("tier_iterations", C.c_int64 * 3),
                ("max_final_residual", C.c_double), ("sum_final_residual", C.c_double),
                ("graph_launches", C.c_int64), ("autotune_trials", C.c_int64), ("tc_gemm_ms", C.c_double),
                ("tc_bytes", C.c_double), ("tc_flops_by_type", C.c_double * 4),
                ("tc_gemm_ms_by_type", C.c_double * 4), ("tc_build_ms", C.c_double),
                ("tc_build_phase_ms", C.c_double * 5), ("enlarge_host_ms", C.c_double), ("diag_ms", C.c_double),
                ("truncate_rho_ms", C.c_double), ("truncate_eig_ms", C.c_double), ("env_wall_ms", C.c_double),
                ("tc_stage_alg_bytes", C.c_double * 2), ("tc_stage_box_bytes", C.c_double * 4),
                ("tc_stage_dense_bytes", C.c_double * 4), ("tc_gemm_ms_by_stage", C.c_double * 2),
                ("davidson_iterations", C.c_int64), ("inner_matvecs", C.c_int64), ("n_solves", C.c_int64),
                ("n_solves_above_tol", C.c_int64), ("sweep_max_residual", C.c_double),
                ("enlarge_dev_ms", C.c_double), ("enlarge_bytes", C.c_double),
                ("rdm_ms", C.c_double), ("rdm_env_bytes", C.c_double), ("h2d_wait_ms", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for k in ("tier_iterations", "tc_flops_by_type", "tc_gemm_ms_by_type", "tc_build_phase_ms",
                  "tc_stage_alg_bytes", "tc_stage_box_bytes", "tc_stage_dense_bytes",
                  "tc_gemm_ms_by_stage"):
            d[k] = list(d[k])
        return d


_lib = None


def lib():
    """Load libgbdmrg.so (built by paper_2609_09990_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2609_09990_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "gbd_create": (C.c_int, [C.POINTER(vp), C.c_int]),
        "gbd_destroy": (None, [vp]),
        "gbd_last_error": (C.c_char_p, [vp]),
        "gbd_solve": (C.c_int, [vp, C.POINTER(gbd_problem), C.POINTER(gbd_schedule), C.POINTER(gbd_result)]),
        "gbd_setup": (C.c_int, [vp, C.POINTER(gbd_problem), C.POINTER(gbd_schedule)]),
        "gbd_solve_states": (C.c_int, [vp, C.POINTER(gbd_problem), C.POINTER(gbd_schedule), C.c_int32, C.c_double,
                                        C.c_double, C.c_int32, C.POINTER(gbd_result), _dp, _ip]),
        "gbd_solve_batched": (C.c_int, [vp, C.c_int32, C.POINTER(gbd_problem), C.POINTER(gbd_schedule),
                                        C.POINTER(gbd_result)]),
        "gbd_set_batch_workers": (C.c_int, [vp, C.c_int32]),
        "gbd_host_batch_costs": (C.c_int, [C.c_int32, C.POINTER(gbd_problem), C.POINTER(gbd_schedule), _dp]),
        "gbd_host_partition": (C.c_int, [C.c_int32, _dp, C.c_int32, _ip, _dp]),
        "gbd_set_graphs": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tc_min_two_site": (C.c_int, [vp, C.c_int64]),
        "gbd_set_accurate_tier": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tier_stop": (C.c_int, [vp, C.c_double, C.c_int32]),
        "gbd_set_env_precision": (C.c_int, [vp, C.c_int32]),
        "gbd_gemm_tc_selftest": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                           C.c_uint64, _dp, _dp]),
        "gbd_set_preconditioner": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tc_tile": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tc_order": (C.c_int, [vp, C.c_int32]),
        "gbd_probe_step": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, _dp, _dp, _dp]),
        "gbd_init_state": (C.c_int, [vp]),
        "gbd_save_state": (C.c_int, [vp]),
        "gbd_pcg_selftest": (C.c_int, [vp, C.c_int32, _dp, _dp, C.c_double, _dp, C.POINTER(C.c_int64)]),
        "gbd_restore_state": (C.c_int, [vp]),
        "gbd_set_sweep_schedule": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_double]),
        "gbd_set_precision": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "gbd_run_sweep": (C.c_int, [vp, C.c_int32, _dp]),
        "gbd_final_energy": (C.c_int, [vp, _dp]),
        "gbd_get_bond": (C.c_int, [vp, C.c_int32, _ip, C.c_int32, _ip]),
        "gbd_set_mps": (C.c_int, [vp, _ip, _ip, _dp, C.c_int32]),
        "gbd_two_site_size": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int64)]),
        "gbd_apply_heff": (C.c_int, [vp, C.c_int32, _dp, _dp, _dp]),
        "gbd_apply_heff_prec": (C.c_int, [vp, C.c_int32, C.c_int32, _dp, _dp]),
        "gbd_run_step": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, _dp, _dp, _dp,
                                   C.c_int32, _ip]),
        "gbd_rdms": (C.c_int, [vp, _dp, _dp]),
        "gbd_rdms_ci": (C.c_int, [vp, _dp, _dp]),
        "gbd_set_env_conjugates": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tc_order_a": (C.c_int, [vp, C.c_int32]),
        "gbd_set_tc_sout_split": (C.c_int, [vp, C.c_int32]),
        "gbd_host_mpo_conjugates": (C.c_int, [C.c_int32, _dp, C.c_int32, _dp, C.c_int32, C.c_int32, C.c_int32, _ip,
                                              _ip, C.c_int32, _ip]),
        "gbd_env_conjugates": (C.c_int, [vp, C.c_int32, C.c_int32, _ip, _ip, C.c_int32, _ip]),
        "gbd_orbital_rdms_ci": (C.c_int, [vp, _dp, _dp]),
        "gbd_rdm3": (C.c_int, [vp, _dp]),
        "gbd_orbital_rdms": (C.c_int, [vp, _dp, _dp]),
        "gbd_orbital_entropies": (C.c_int, [vp, _dp, _dp]),
        "gbd_mi_order": (C.c_int, [vp, C.POINTER(gbd_problem), C.POINTER(gbd_schedule), _ip, _dp]),
        "gbd_mpo_labels": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_uint64), C.c_int32, _ip]),
        "gbd_env_block": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp, C.c_int64, _ip, _ip]),
        "gbd_get_stats": (C.c_int, [vp, C.POINTER(gbd_stats)]),
        "gbd_get_batch_stats": (C.c_int, [vp, C.POINTER(gbd_stats)]),
        "gbd_mps_init_value": (C.c_double, [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int32]),
        "gbd_wait_selftest": (C.c_int, [C.c_int32, C.c_int32, _ip, _ip]),
        "gbd_correction_selftest": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _dp, _dp, _dp, C.c_double, _dp, _dp,
                                               _dp]),
        "gbd_tc_selftest": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                      _dp, _dp]),
        "gbd_tc_rate": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp, _dp]),
        "gbd_multi_dot": (C.c_int, [vp, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, _dp]),
        "gbd_multi_dot_noalloc": (C.c_int, [C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.c_void_p]),
        "gbd_train_precond": (C.c_int, [vp, C.c_int32, C.POINTER(gbd_problem), C.POINTER(gbd_schedule), C.c_int32,
                                        C.c_double, _dp]),
        "gbd_save_precond": (C.c_int, [vp, C.c_char_p]),
        "gbd_load_precond": (C.c_int, [vp, C.c_char_p]),
        "gbd_set_precond_weights": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "gbd_mlp_loss_grad": (C.c_int, [vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                        C.c_int64, C.POINTER(C.c_float), C.c_double, _dp, _dp]),
        "gbd_mlp_precond": (C.c_int, [vp, _dp, _dp, C.c_double, C.c_double, C.c_int64, _dp]),
        "gbd_davidson_counts": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "gbd_host_sym_eig": (C.c_int, [C.c_int32, _dp, _dp, _dp]),
        "gbd_host_fiedler_order": (C.c_int, [C.c_int32, _dp, _ip]),
        "gbd_host_initial_dims": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _ip, _ip, C.c_int32]),
        "gbd_host_select": (C.c_int, [C.c_int32, _dp, _ip, _ip, C.c_int32, C.c_double, C.c_double, C.c_double,
                                      C.c_int32, _ip, _ip, _dp]),
        "gbd_set_adaptive_bond_dim": (C.c_int, [vp, C.c_double, C.c_int32]),
        "gbd_host_mpo": (C.c_int, [C.c_int32, _dp, C.c_int32, _dp, C.c_int32, _ip, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


class GbdError(RuntimeError):
    pass


class Context:
    """Owns one gbd_ctx (device memory, stream) and keeps the marshalled
    inputs alive while the library reads them."""

    def __init__(self, device: int = 0):
        self.L = lib()
        self.ptr = C.c_void_p()
        rc = self.L.gbd_create(C.byref(self.ptr), device)
        if rc != GBD_OK:
            raise GbdError(f"gbd_create failed: {ERRORS.get(rc, rc)}")
        self._keep = []

    def last_error(self):
        return self.L.gbd_last_error(self.ptr).decode(errors="replace")

    def close(self):
        if self.ptr:
            self.L.gbd_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != GBD_OK:
            msg = self.L.gbd_last_error(self.ptr).decode()
            raise GbdError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")

    def _structs(self, *args, **kw):
        p, s, self._keep = _make_structs(*args, **kw)
        return p, s

    def solve(self, h, chol, n_elec, two_sz, bond_dims, tols, rdms=False, **kw):
        """gbd_solve; returns dict(energy, sweep_energies, rdm1, rdm2, ...)."""
        p, s = self._structs(h, chol, n_elec, two_sz, bond_dims, tols, **kw)
        n = p.n_orb
        se = np.zeros(len(bond_dims))
        r1 = np.zeros((n, n)) if rdms else None
        r2 = np.zeros((n, n, n, n)) if rdms else None
        res = gbd_result(0.0, _d(se), _d(r1), _d(r2), 0.0, 0, 0)
        self._check(self.L.gbd_solve(self.ptr, C.byref(p), C.byref(s), C.byref(res)), "gbd_solve")
        return dict(energy=res.energy, sweep_energies=se, rdm1=r1, rdm2=r2,
                    max_discarded_weight=res.max_discarded_weight, n_matvec=res.n_matvec)

    def solve_batched(self, problems, rdms=False, workers=0, check=True):
        """gbd_solve_batched over a list of (h, chol, n_elec, two_sz, bond_dims, tols, kwargs); returns
        (return code, list of result dicts with their own status)."""
        n = len(problems)
        ps = (gbd_problem * max(n, 1))()
        ss = (gbd_schedule * max(n, 1))()
        rs = (gbd_result * max(n, 1))()
        keep, outs = [], []
        for i, (h, chol, ne, sz, bd, tl, kw) in enumerate(problems):
            p, s = self._structs(h, chol, ne, sz, bd, tl, **kw)
            keep.append(self._keep)
            ps[i] = p
            ss[i] = s
            no = p.n_orb
            se = np.zeros(len(bd))
            r1 = np.zeros((no, no)) if rdms else None
            r2 = np.zeros((no, no, no, no)) if rdms else None
            outs.append((se, r1, r2))
            rs[i] = gbd_result(0.0, _d(se), _d(r1), _d(r2), 0.0, 0, 0)
        self._check(self.L.gbd_set_batch_workers(self.ptr, workers), "gbd_set_batch_workers")
        rc = self.L.gbd_solve_batched(self.ptr, n, ps, ss, rs)
        if check:
            self._check(rc, "gbd_solve_batched")
        res = [dict(energy=rs[i].energy, sweep_energies=outs[i][0], rdm1=outs[i][1], rdm2=outs[i][2],
                    max_discarded_weight=rs[i].max_discarded_weight, n_matvec=rs[i].n_matvec,
                    status=rs[i].status) for i in range(n)]
        return rc, res

    def solve_states(self, h, chol, n_elec, two_sz, bond_dims, tols, n_states, penalty=5.0, target_s2=0.0,
                     max_extra=2, rdms=False, check=True, **kw):
        """gbd_solve_states: (return code, list of result dicts with 's2', one per root found)."""
        p, s = self._structs(h, chol, n_elec, two_sz, bond_dims, tols, **kw)
        n = p.n_orb
        rs = (gbd_result * n_states)()
        outs = []
        for i in range(n_states):
            se = np.zeros(len(bond_dims))
            r1 = np.zeros((n, n)) if rdms else None
            r2 = np.zeros((n, n, n, n)) if rdms else None
            outs.append((se, r1, r2))
            rs[i] = gbd_result(0.0, _d(se), _d(r1), _d(r2), 0.0, 0, 0)
        s2 = np.zeros(n_states)
        nf = C.c_int32(0)
        rc = self.L.gbd_solve_states(self.ptr, C.byref(p), C.byref(s), n_states, float(penalty), float(target_s2),
                                     max_extra, rs, _d(s2), C.byref(nf))
        if check:
            self._check(rc, "gbd_solve_states")
        res = [dict(energy=rs[i].energy, sweep_energies=outs[i][0], rdm1=outs[i][1], rdm2=outs[i][2],
                    s2=float(s2[i]), n_matvec=rs[i].n_matvec) for i in range(nf.value)]
        return rc, res

    def setup(self, h, chol, n_elec, two_sz, bond_dims, tols, **kw):
        p, s = self._structs(h, chol, n_elec, two_sz, bond_dims, tols, **kw)
        self._check(self.L.gbd_setup(self.ptr, C.byref(p), C.byref(s)), "gbd_setup")

    def set_precision(self, precision, fp64_refine=2):
        self._check(self.L.gbd_set_precision(self.ptr, precision, fp64_refine), "gbd_set_precision")

    def init_state(self):
        self._check(self.L.gbd_init_state(self.ptr), "gbd_init_state")

    def pcg_selftest(self, k, x, r, theta):
        """(t, matvecs) of the solver's inner-PCG correction at centre k."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        t = np.empty_like(x)
        mv = C.c_int64()
        self._check(self.L.gbd_pcg_selftest(self.ptr, k, _d(x), _d(r), float(theta), _d(t), C.byref(mv)),
                    "gbd_pcg_selftest")
        return t, mv.value

    def save_state(self):
        self._check(self.L.gbd_save_state(self.ptr), "gbd_save_state")

    def restore_state(self):
        self._check(self.L.gbd_restore_state(self.ptr), "gbd_restore_state")

    def set_sweep_schedule(self, sweep, M, tol):
        self._check(self.L.gbd_set_sweep_schedule(self.ptr, sweep, M, tol), "gbd_set_sweep_schedule")

    def run_sweep(self, sweep):
        e = C.c_double()
        self._check(self.L.gbd_run_sweep(self.ptr, sweep, C.byref(e)), "gbd_run_sweep")
        return e.value

    def final_energy(self):
        e = C.c_double()
        self._check(self.L.gbd_final_energy(self.ptr, C.byref(e)), "gbd_final_energy")
        return e.value

    def get_bond(self, bond):
        cnt = C.c_int32()
        self._check(self.L.gbd_get_bond(self.ptr, bond, None, 0, C.byref(cnt)), "gbd_get_bond")
        t = np.zeros(3 * cnt.value, dtype=np.int32)
        self._check(self.L.gbd_get_bond(self.ptr, bond, _i(t), cnt.value, C.byref(cnt)), "gbd_get_bond")
        return t.reshape(-1, 3)

    def set_mps(self, n_sectors, sectors, data, center):
        ns = np.ascontiguousarray(n_sectors, dtype=np.int32)
        sc = np.ascontiguousarray(sectors, dtype=np.int32)
        dt = np.ascontiguousarray(data, dtype=np.float64)
        self._check(self.L.gbd_set_mps(self.ptr, _i(ns), _i(sc), _d(dt), center), "gbd_set_mps")

    def two_site_size(self, k):
        n = C.c_int64()
        self._check(self.L.gbd_two_site_size(self.ptr, k, C.byref(n)), "gbd_two_site_size")
        return n.value

    def apply_heff(self, k, x, want_diag=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        d = np.zeros_like(x) if want_diag else None
        self._check(self.L.gbd_apply_heff(self.ptr, k, _d(x), _d(y), _d(d)), "gbd_apply_heff")
        return (y, d) if want_diag else y

    def apply_heff_prec(self, k, x, prec):
        """H_eff x through the tensor-core sigma (prec 1 TF32, 2 BF16, 3 TF32x3, 4 BF16x3)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        self._check(self.L.gbd_apply_heff_prec(self.ptr, k, prec, _d(x), _d(y)), "gbd_apply_heff_prec")
        return y

    def set_tc_tile(self, ncap):
        self._check(self.L.gbd_set_tc_tile(self.ptr, ncap), "gbd_set_tc_tile")

    def set_adaptive_bond_dim(self, max_discarded, m_min=1):
        """Per-bond adaptive bond dimension (0 = fixed M) for the following solves."""
        self._check(self.L.gbd_set_adaptive_bond_dim(self.ptr, float(max_discarded), int(m_min)),
                    "gbd_set_adaptive_bond_dim")

    def set_tc_order(self, order):
        self._check(self.L.gbd_set_tc_order(self.ptr, order), "gbd_set_tc_order")

    def set_tc_sout_split(self, min_rows):
        self._check(self.L.gbd_set_tc_sout_split(self.ptr, min_rows), "gbd_set_tc_sout_split")

    def set_tc_order_a(self, order):
        self._check(self.L.gbd_set_tc_order_a(self.ptr, order), "gbd_set_tc_order_a")

    def set_preconditioner(self, preconditioner):
        self._check(self.L.gbd_set_preconditioner(self.ptr, preconditioner), "gbd_set_preconditioner")

    def set_env_precision(self, prec):
        """Environment updates of the steps: 0 FP64, 3 TF32x3, 4 BF16x3 (tensor cores)."""
        self._check(self.L.gbd_set_env_precision(self.ptr, prec), "gbd_set_env_precision")

    def gemm_tc_selftest(self, M, N, K, nterms, flags, prec=3, seed=1):
        """(max |tensor-core - FP64|, max |FP64|) of a random grouped GEMM plan."""
        e, r = C.c_double(), C.c_double()
        self._check(self.L.gbd_gemm_tc_selftest(self.ptr, M, N, K, nterms, flags, prec, seed, C.byref(e),
                                                C.byref(r)), "gbd_gemm_tc_selftest")
        return e.value, r.value

    def set_tier_stop(self, floor_mult, hard_stag=0):
        self._check(self.L.gbd_set_tier_stop(self.ptr, float(floor_mult), int(hard_stag)), "gbd_set_tier_stop")

    def set_accurate_tier(self, prec):
        """3 = TF32x3 (default), 4 = BF16x3."""
        self._check(self.L.gbd_set_accurate_tier(self.ptr, prec), "gbd_set_accurate_tier")

    def set_tc_min_two_site(self, n):
        self._check(self.L.gbd_set_tc_min_two_site(self.ptr, n), "gbd_set_tc_min_two_site")

    def set_graphs(self, enable):
        self._check(self.L.gbd_set_graphs(self.ptr, 1 if enable else 0), "gbd_set_graphs")

    def probe_step(self, k, precision, fp64_refine, tol):
        """(Ritz value, FP64 Rayleigh quotient, FP64 residual) of one Davidson solve at centre k."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(self.L.gbd_probe_step(self.ptr, k, precision, fp64_refine, tol, C.byref(a), C.byref(b),
                                          C.byref(c)), "gbd_probe_step")
        return a.value, b.value, c.value

    def run_step(self, k, direction, M, tol):
        e, tau, nk = C.c_double(), C.c_double(), C.c_int32()
        kept = np.zeros(max(M, 1))
        self._check(self.L.gbd_run_step(self.ptr, k, direction, M, tol, C.byref(e), C.byref(tau), _d(kept),
                                        len(kept), C.byref(nk)), "gbd_run_step")
        return e.value, tau.value, kept[:nk.value].copy()

    def rdms(self, n):
        r1 = np.zeros((n, n))
        r2 = np.zeros((n, n, n, n))
        self._check(self.L.gbd_rdms(self.ptr, _d(r1), _d(r2)), "gbd_rdms")
        return r1, r2

    def set_env_conjugates(self, enable):
        self._check(self.L.gbd_set_env_conjugates(self.ptr, int(enable)), "gbd_set_env_conjugates")

    def env_conjugates(self, side, bond):
        """gbd_env_conjugates: (partner, sign) arrays of one bond."""
        cnt = C.c_int32(0)
        self._check(self.L.gbd_env_conjugates(self.ptr, side, bond, None, None, 0, C.byref(cnt)),
                    "gbd_env_conjugates")
        part = np.zeros(cnt.value, dtype=np.int32)
        sg = np.zeros(cnt.value, dtype=np.int32)
        self._check(self.L.gbd_env_conjugates(self.ptr, side, bond, _i(part), _i(sg), cnt.value, C.byref(cnt)),
                    "gbd_env_conjugates")
        return part, sg

    def rdms_ci(self, n):
        """gbd_rdms_ci: the same RDMs from the determinant expansion."""
        r1 = np.zeros((n, n))
        r2 = np.zeros((n, n, n, n))
        self._check(self.L.gbd_rdms_ci(self.ptr, _d(r1), _d(r2)), "gbd_rdms_ci")
        return r1, r2

    def rdm3(self, n):
        """gbd_rdm3: the spin-summed 3-RDM [n]*6 of the current state."""
        out = np.zeros((n,) * 6)
        self._check(self.L.gbd_rdm3(self.ptr, _d(out)), "gbd_rdm3")
        return out

    def orbital_rdms(self, n):
        """gbd_orbital_rdms: (rho1 [n,4,4], rho2 [n(n-1)/2,16,16])."""
        r1 = np.zeros((n, 4, 4))
        r2 = np.zeros((max(n * (n - 1) // 2, 1), 16, 16))
        self._check(self.L.gbd_orbital_rdms(self.ptr, _d(r1), _d(r2)), "gbd_orbital_rdms")
        return r1, r2[:n * (n - 1) // 2]

    def orbital_rdms_ci(self, n):
        """gbd_orbital_rdms_ci: the same from the determinant expansion."""
        r1 = np.zeros((n, 4, 4))
        r2 = np.zeros((max(n * (n - 1) // 2, 1), 16, 16))
        self._check(self.L.gbd_orbital_rdms_ci(self.ptr, _d(r1), _d(r2)), "gbd_orbital_rdms_ci")
        return r1, r2[:n * (n - 1) // 2]

    def orbital_entropies(self, n):
        """gbd_orbital_entropies: (s1 [n], mutual information [n,n])."""
        s1 = np.zeros(n)
        mi = np.zeros((n, n))
        self._check(self.L.gbd_orbital_entropies(self.ptr, _d(s1), _d(mi)), "gbd_orbital_entropies")
        return s1, mi

    def mi_order(self, h, chol, n_elec, two_sz, bond_dims, tols, **kw):
        """gbd_mi_order: (order, mutual information) from a preliminary solve."""
        p, s = self._structs(h, chol, n_elec, two_sz, bond_dims, tols, **kw)
        n = p.n_orb
        order = np.zeros(n, dtype=np.int32)
        mi = np.zeros((n, n))
        self._check(self.L.gbd_mi_order(self.ptr, C.byref(p), C.byref(s), _i(order), _d(mi)), "gbd_mi_order")
        return order, mi

    def mpo_labels(self, bond):
        cnt = C.c_int32()
        self._check(self.L.gbd_mpo_labels(self.ptr, bond, None, 0, C.byref(cnt)), "gbd_mpo_labels")
        k = np.zeros(cnt.value, dtype=np.uint64)
        self._check(self.L.gbd_mpo_labels(self.ptr, bond, k.ctypes.data_as(C.POINTER(C.c_uint64)), cnt.value,
                                          C.byref(cnt)), "gbd_mpo_labels")
        return k

    def env_block(self, side, bond, channel, sector):
        r, c = C.c_int32(), C.c_int32()
        self._check(self.L.gbd_env_block(self.ptr, side, bond, channel, sector, None, 0, C.byref(r),
                                         C.byref(c)), "gbd_env_block")
        out = np.zeros(r.value * c.value)
        self._check(self.L.gbd_env_block(self.ptr, side, bond, channel, sector, _d(out), out.size,
                                         C.byref(r), C.byref(c)), "gbd_env_block")
        return out.reshape(r.value, c.value)

    def multi_dot(self, V_ptr, stride, k, x_ptr, n):
        """out[j] = V_j . x over device pointers (e.g. torch tensor data_ptr())."""
        out = np.zeros(k)
        self._check(self.L.gbd_multi_dot(self.ptr, V_ptr, stride, k, x_ptr, n, _d(out)), "gbd_multi_dot")
        return out

    def train_precond(self, problems, epochs=400, lr=3e-3):
        """problems: list of (h, chol, n_elec, two_sz, bond_dims, tols, kwargs)."""
        ps = (gbd_problem * len(problems))()
        ss = (gbd_schedule * len(problems))()
        keep = []
        for i, (h, chol, ne, sz, bd, tl, kw) in enumerate(problems):
            p, s = self._structs(h, chol, ne, sz, bd, tl, **kw)
            keep.append(self._keep)
            ps[i] = p
            ss[i] = s
        loss = C.c_double()
        self._check(self.L.gbd_train_precond(self.ptr, len(problems), ps, ss, epochs, lr, C.byref(loss)),
                    "gbd_train_precond")
        return loss.value

    def save_precond(self, path):
        self._check(self.L.gbd_save_precond(self.ptr, path.encode()), "gbd_save_precond")

    def load_precond(self, path):
        self._check(self.L.gbd_load_precond(self.ptr, path.encode()), "gbd_load_precond")

    def set_precond_weights(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.L.gbd_set_precond_weights(self.ptr, p.ctypes.data_as(C.POINTER(C.c_float))),
                    "gbd_set_precond_weights")

    def mlp_loss_grad(self, X, y, w, params, lam=0.0):
        fp = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        X, y, w, params = fp(X), fp(y), fp(w), fp(params)
        loss = C.c_double()
        grad = np.zeros(params.size)
        f = C.POINTER(C.c_float)
        self._check(self.L.gbd_mlp_loss_grad(self.ptr, X.ctypes.data_as(f), y.ctypes.data_as(f), w.ctypes.data_as(f),
                                             len(y), params.ctypes.data_as(f), lam, C.byref(loss), _d(grad)),
                    "gbd_mlp_loss_grad")
        return loss.value, grad

    def mlp_precond(self, r, d, theta, it):
        r = np.ascontiguousarray(r, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        t = np.zeros_like(r)
        self._check(self.L.gbd_mlp_precond(self.ptr, _d(r), _d(d), theta, it, len(r), _d(t)), "gbd_mlp_precond")
        return t

    def davidson_counts(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.L.gbd_davidson_counts(self.ptr, C.byref(a), C.byref(b), C.byref(c)), "gbd_davidson_counts")
        return a.value, b.value, c.value

    def stats(self):
        s = gbd_stats()
        self.L.gbd_get_stats(self.ptr, C.byref(s))
        return s.as_dict()

    def batch_stats(self):
        s = gbd_stats()
        self.L.gbd_get_batch_stats(self.ptr, C.byref(s))
        return s.as_dict()


# ---- host-only planner pieces
def _make_structs(h, chol, n_elec, two_sz, bond_dims, tols, seed=1, precision=GBD_FP64,
                  preconditioner=GBD_PRECOND_DIAG, max_iter=100, max_subspace=24, svd_cutoff=1e-12,
                  e_core=0.0, fp64_refine=2):
    """(gbd_problem, gbd_schedule, arrays they point into: keep them alive)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    chol = np.ascontiguousarray(chol, dtype=np.float64)
    bd = np.ascontiguousarray(bond_dims, dtype=np.int32)
    tl = np.ascontiguousarray(tols, dtype=np.float64)
    p = gbd_problem(h.shape[0], n_elec, two_sz, chol.shape[0], _d(h), _d(chol), e_core)
    s = gbd_schedule(len(bd), _i(bd), _d(tl), max_iter, max_subspace, precision, preconditioner,
                     seed, svd_cutoff, fp64_refine)
    return p, s, [h, chol, bd, tl]


def host_batch_costs(problems):
    """gbd_host_batch_costs over (h, chol, n_elec, two_sz, bond_dims, tols, kwargs) tuples."""
    n = len(problems)
    ps = (gbd_problem * max(n, 1))()
    ss = (gbd_schedule * max(n, 1))()
    keep = []
    for i, (h, chol, ne, sz, bd, tl, kw) in enumerate(problems):
        ps[i], ss[i], k = _make_structs(h, chol, ne, sz, bd, tl, **kw)
        keep.append(k)
    cost = np.zeros(max(n, 1))
    rc = lib().gbd_host_batch_costs(n, ps, ss, _d(cost))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_batch_costs: {ERRORS.get(rc, rc)}")
    return cost[:n].copy()


def host_partition(cost, ranks):
    """gbd_host_partition: (owner rank of each problem, summed cost per rank)."""
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    n = cost.size
    owner = np.zeros(max(n, 1), dtype=np.int32)
    load = np.zeros(max(ranks, 1))
    rc = lib().gbd_host_partition(n, _d(cost), ranks, _i(owner), _d(load))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_partition: {ERRORS.get(rc, rc)}")
    return owner[:n].copy(), load[:ranks].copy()


def host_sym_eig(A):
    """Host eigensolver of the decimation: (w ascending, Z columns = eigenvectors)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, n))
    rc = lib().gbd_host_sym_eig(n, _d(A), _d(w), _d(Z))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_sym_eig: {ERRORS.get(rc, rc)}")
    return w, Z


def fiedler_order(W):
    """gbd_host_fiedler_order: orbital order (order[k] = orbital at site k) from couplings W."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    n = W.shape[0]
    order = np.zeros(max(n, 1), dtype=np.int32)
    rc = lib().gbd_host_fiedler_order(n, _d(W), _i(order))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_fiedler_order: {ERRORS.get(rc, rc)}")
    return order[:n].copy()


def host_initial_dims(n, n_alpha, n_beta, M):
    L = lib()
    ns = np.zeros(n + 1, dtype=np.int32)
    cap = 8192
    tr = np.zeros(3 * cap, dtype=np.int32)
    rc = L.gbd_host_initial_dims(n, n_alpha, n_beta, M, _i(ns), _i(tr), cap)
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_initial_dims: {ERRORS.get(rc, rc)}")
    out, pos = [], 0
    for k in range(n + 1):
        d = {}
        for _ in range(ns[k]):
            d[(int(tr[pos]), int(tr[pos + 1]))] = int(tr[pos + 2])
            pos += 3
        out.append(d)
    return out


def host_select(lam, key, j, M, cutoff=1e-12, tie=1e-10, max_discarded=0.0, m_min=1):
    L = lib()
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    key = np.ascontiguousarray(key, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    idx = np.zeros(max(len(lam), 1), dtype=np.int32)
    nk = C.c_int32()
    tot = C.c_double()
    rc = L.gbd_host_select(len(lam), _d(lam), _i(key), _i(j), M, cutoff, tie, float(max_discarded), int(m_min),
                           _i(idx), C.byref(nk), C.byref(tot))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_select: {ERRORS.get(rc, rc)}")
    return idx[:nk.value].copy(), tot.value


def host_mpo(h, chol, k_switch=None, dense=False):
    L = lib()
    h = np.ascontiguousarray(h, dtype=np.float64)
    chol = np.ascontiguousarray(chol, dtype=np.float64)
    n = h.shape[0]
    bd = np.zeros(n + 1, dtype=np.int32)
    out = np.zeros((4 ** n, 4 ** n)) if dense else None
    rc = L.gbd_host_mpo(n, _d(h), chol.shape[0], _d(chol), n // 2 if k_switch is None else k_switch, _i(bd), _d(out))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_mpo: {ERRORS.get(rc, rc)}")
    return (bd, out) if dense else bd


def host_mpo_conjugates(h, chol, side, bond, k_switch=None):
    """gbd_host_mpo_conjugates: (partner, sign) of the certified conjugate
    channel pairs of one bond of the MPO of (h, chol)."""
    L = lib()
    h = np.ascontiguousarray(h, dtype=np.float64)
    chol = np.ascontiguousarray(chol, dtype=np.float64)
    n = h.shape[0]
    ks = n // 2 if k_switch is None else k_switch
    cnt = C.c_int32(0)
    rc = L.gbd_host_mpo_conjugates(n, _d(h), chol.shape[0], _d(chol), ks, side, bond, None, None, 0, C.byref(cnt))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_mpo_conjugates: {ERRORS.get(rc, rc)}")
    part = np.zeros(cnt.value, dtype=np.int32)
    sg = np.zeros(cnt.value, dtype=np.int32)
    rc = L.gbd_host_mpo_conjugates(n, _d(h), chol.shape[0], _d(chol), ks, side, bond, _i(part), _i(sg), cnt.value,
                                   C.byref(cnt))
    if rc != GBD_OK:
        raise GbdError(f"gbd_host_mpo_conjugates: {ERRORS.get(rc, rc)}")
    return part, sg


def multi_dot_noalloc(device, V_ptr, stride, k, x_ptr, n, out_ptr, stream=None):
    """gbd_multi_dot_noalloc: out[j] = V_j . x into the device array out_ptr,
    enqueued on `stream` (a raw cudaStream_t value or None); no allocation."""
    rc = lib().gbd_multi_dot_noalloc(device, V_ptr, stride, k, x_ptr, n, out_ptr, stream)
    if rc != GBD_OK:
        raise GbdError(f"gbd_multi_dot_noalloc: {ERRORS.get(rc, rc)}")


def tc_selftest(prec, M, N, K, nterms, seed=1, device=0):
    """(max |error|, max |reference|) of the tensor-core grouped GEMM self-test."""
    e, r = C.c_double(), C.c_double()
    rc = lib().gbd_tc_selftest(device, prec, M, N, K, nterms, seed, C.byref(e), C.byref(r))
    if rc != GBD_OK:
        raise GbdError(f"gbd_tc_selftest: {ERRORS.get(rc, rc)}")
    return e.value, r.value


def correction_selftest(kind, x, sx, diag, theta, device=0):
    """(r, t, |r|^2) of one Davidson correction on the device (kind: GBD_PRECOND_DIAG or _OLSEN)."""
    x, sx, diag = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, sx, diag))
    n = x.size
    r, t, rr = np.empty(n), np.empty(n), C.c_double()
    rc = lib().gbd_correction_selftest(device, kind, n, _d(x), _d(sx), _d(diag), float(theta), _d(r), _d(t),
                                       C.byref(rr))
    if rc != GBD_OK:
        raise GbdError(f"gbd_correction_selftest: {ERRORS.get(rc, rc)}")
    return r, t, rr.value


def tc_rate(prec, M, N, K, reps=10, device=0):
    """(TFLOP/s, ms per launch) of one dense M x N x K tensor-core product."""
    t, m = C.c_double(), C.c_double()
    rc = lib().gbd_tc_rate(device, prec, M, N, K, reps, C.byref(t), C.byref(m))
    if rc != GBD_OK:
        raise GbdError(f"gbd_tc_rate: {ERRORS.get(rc, rc)}")
    return t.value, m.value


def wait_selftest(arrive, device=0):
    """(error flag, waited_ok) of one bounded mbarrier wait; arrive=False lets it run out."""
    e, o = C.c_int32(), C.c_int32()
    rc = lib().gbd_wait_selftest(device, 1 if arrive else 0, C.byref(e), C.byref(o))
    if rc != GBD_OK:
        raise GbdError(f"gbd_wait_selftest: {ERRORS.get(rc, rc)}")
    return e.value, o.value


def mps_init_value(seed, site, na, nb, s, row, col):
    return lib().gbd_mps_init_value(seed, site, na, nb, s, row, col)
