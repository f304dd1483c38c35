"""Python binding of libmlsd (include/mlsd.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
numpy arrays and torch tensors to pointers and C structs and checks return
codes.  Importing it fails loudly when the library has not been built: there
is no fallback implementation.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlsd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmlsd.so is not built ({LIB_PATH}); run __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

MLSD_FP32, MLSD_FP64 = 0, 1
MLSD_PLAIN, MLSD_SURROGATE = 0, 1
ERRORS = {0: "MLSD_OK", -1: "MLSD_EINVAL", -2: "MLSD_ENOMEM", -3: "MLSD_ECUDA",
          -4: "MLSD_ETIMEOUT", -5: "MLSD_ENONFINITE", -6: "MLSD_EUNSUPPORTED"}
EXPORTED = ["mlsd_build_levels", "mlsd_free_levels", "mlsd_level_info", "mlsd_solve_level",
            "mlsd_offdiag", "mlsd_effective_diffusivity", "mlsd_status", "mlsd_macro_step",
            "mlsd_macro_dt", "mlsd_grid_psi", "mlsd_dns_run", "mlsd_coarse_grain",
            "mlsd_level_work", "mlsd_corrector_energy", "mlsd_launch_count", "mlsd_profile", "mlsd_profile_collect",
            "mlsd_coarse_grain_noalloc", "mlsd_dns_dt", "mlsd_patch_sizes",
            "mlsd_macro_step_dirichlet", "mlsd_dns_run_dirichlet", "mlsd_check_wait_timeout",
            "mlsd_dns_status", "mlsd_dns_kernel",
            "mlsd_surrogate_param_count", "mlsd_surrogate_create", "mlsd_surrogate_free",
            "mlsd_surrogate_set_params", "mlsd_surrogate_get_params", "mlsd_surrogate_features",
            "mlsd_surrogate_grad", "mlsd_surrogate_train_step", "mlsd_surrogate_predict",
            "mlsd_solve_level_surrogate", "mlsd_surrogate_set_engine", "mlsd_surrogate_status",
            "mlsd_surrogate_dataset", "mlsd_surrogate_train", "mlsd_surrogate_save",
            "mlsd_surrogate_load", "mlsd_attach_surrogate", "mlsd_surrogate_fallbacks",
            "mlsd_surrogate_symmetry", "mlsd_strerror"]
SUR_CUDA, SUR_TENSOR = 0, 1
SUR_IN, SUR_FEATURES = 640, 606
SUR_PSI_SCALE, SUR_T_SCALE, SUR_Y_SCALE, SUR_GAP_WEIGHT = 32.0, 10.0, 300.0, 0.3
NOALLOC_MAX_MACRO = 256


class MlsdError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.mlsd_strerror(code).decode()
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class mlsd_problem(ctypes.Structure):
    _fields_ = [("n_macro", ctypes.c_int), ("kappa", ctypes.c_double), ("n_modes", ctypes.c_int),
                ("k1", ctypes.c_void_p), ("k2", ctypes.c_void_p), ("re", ctypes.c_void_p),
                ("im", ctypes.c_void_p), ("n_levels", ctypes.c_int),
                ("band_edges", ctypes.c_void_p), ("patch_div", ctypes.c_void_p),
                ("patch_n", ctypes.c_void_p), ("cfl", ctypes.c_double),
                ("t_burn_tau", ctypes.c_double), ("t_avg_tau", ctypes.c_double),
                ("n_burn_fixed", ctypes.c_int64), ("n_avg_fixed", ctypes.c_int64),
                ("precision", ctypes.c_int), ("patch_n_map", ctypes.c_void_p),
                ("n_min", ctypes.c_int), ("n_max", ctypes.c_int), ("periodize", ctypes.c_int)]


class mlsd_level_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("Nl", ctypes.c_int64), ("L", ctypes.c_double),
                ("h", ctypes.c_double), ("n_patches", ctypes.c_int64),
                ("n_diag_modes", ctypes.c_int), ("n_off12_modes", ctypes.c_int),
                ("n_off21_modes", ctypes.c_int), ("tile_bx", ctypes.c_int),
                ("tile_by", ctypes.c_int), ("threads", ctypes.c_int), ("packed", ctypes.c_int),
                ("cluster", ctypes.c_int), ("min_ctas", ctypes.c_int), ("split", ctypes.c_int),
                ("n_classes", ctypes.c_int), ("coef_tmem", ctypes.c_int),
                ("level_launch", ctypes.c_int)]


_P, _I, _D, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_lib.mlsd_build_levels.argtypes = [ctypes.POINTER(mlsd_problem), _P, ctypes.POINTER(_P)]
_lib.mlsd_free_levels.argtypes = [_P]
_lib.mlsd_free_levels.restype = None
_lib.mlsd_level_info.argtypes = [_P, _I, ctypes.POINTER(mlsd_level_desc)]
_lib.mlsd_solve_level.argtypes = [_P, _I, _P, _P, _P, _P]
_lib.mlsd_offdiag.argtypes = [_P, _I, _P, _P, _P]
_lib.mlsd_effective_diffusivity.argtypes = [_P, _I, _P, _P, _P]
_lib.mlsd_status.argtypes = [_P, _P]
_lib.mlsd_macro_step.argtypes = [_I, _P, _I, _P, _D, _I, _P, _P]
_lib.mlsd_macro_dt.argtypes = [_I, _P, _D, ctypes.POINTER(_D), _P]
_lib.mlsd_grid_psi.argtypes = [_I, _P, _P, _P, _P, _I, _P, _P]
_lib.mlsd_dns_run.argtypes = [_I, _P, _P, _P, _D, _D, _I, _P]
_lib.mlsd_coarse_grain.argtypes = [_I, _P, _I, _P, _P, _P]
_lib.mlsd_level_work.argtypes = [_P, _I, ctypes.POINTER(_L), ctypes.POINTER(_L), ctypes.POINTER(_L), _P]
_lib.mlsd_corrector_energy.argtypes = [_P, _I, _P, _P, _P, _P, _P]
_lib.mlsd_profile.argtypes = [_P, _I]
_lib.mlsd_profile_collect.argtypes = [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_L)]
_lib.mlsd_profile_collect_classes.argtypes = [_P, _I, _I, _P, _P, _P, ctypes.POINTER(ctypes.c_int32)]
_lib.mlsd_level_schedule.argtypes = [_P, _P, _I, _I, _L, _P, ctypes.POINTER(_L)]
_lib.mlsd_launch_count.argtypes = []
_lib.mlsd_launch_count.restype = _L
_lib.mlsd_patch_sizes.argtypes = [_P, _I, _P]
_lib.mlsd_dns_dt.argtypes = [_I, _P, _D, _D, ctypes.POINTER(_D), _P]
_lib.mlsd_macro_step_dirichlet.argtypes = [_I, _P, _I, _P, _D, _I, _D, _D, _P, _P]
_lib.mlsd_dns_run_dirichlet.argtypes = [_I, _P, _P, _P, _I, _D, _D, _I, _D, _D, _P]
_lib.mlsd_check_wait_timeout.argtypes = [_P, _I, _P]
_lib.mlsd_dns_status.argtypes = [_P]
_lib.mlsd_dns_kernel.argtypes = []
_lib.mlsd_dns_kernel.restype = ctypes.c_char_p
_lib.mlsd_coarse_grain_noalloc.argtypes = [_I, _P, _I, _P, _P, _P]
_lib.mlsd_surrogate_param_count.argtypes = [_I]
_lib.mlsd_surrogate_param_count.restype = _L
_lib.mlsd_surrogate_create.argtypes = [_I, _I, _I, ctypes.POINTER(_P)]
_lib.mlsd_surrogate_free.argtypes = [_P]
_lib.mlsd_surrogate_free.restype = None
_lib.mlsd_surrogate_set_params.argtypes = [_P, _I, _P]
_lib.mlsd_surrogate_get_params.argtypes = [_P, _I, _P]
_lib.mlsd_surrogate_features.argtypes = [_P, _I, _P, _P, _P, _P]
_lib.mlsd_surrogate_grad.argtypes = [_P, _I, _P, _P, _I, _P, ctypes.POINTER(_D), _P]
_lib.mlsd_surrogate_train_step.argtypes = [_P, _I, _P, _P, _I, ctypes.c_float, ctypes.POINTER(_D), _P]
_lib.mlsd_surrogate_predict.argtypes = [_P, _P, _L, _P, _P]
_lib.mlsd_solve_level_surrogate.argtypes = [_P, _P, _I, _P, _P, _D, ctypes.POINTER(_L), _P]
_lib.mlsd_surrogate_set_engine.argtypes = [_P, _I]
_lib.mlsd_surrogate_dataset.argtypes = [_P, _I, _P, _P, _P, _P]
_lib.mlsd_surrogate_train.argtypes = [_P, _P, _P, _L, _I, _I, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_uint64, _I, _P, _P]
_lib.mlsd_surrogate_symmetry.argtypes = [_P, _P, _L, _I, _P, _P, _P]
_lib.mlsd_surrogate_save.argtypes = [_P, ctypes.c_char_p]
_lib.mlsd_attach_surrogate.argtypes = [_P, _I, _P, _D]
_lib.mlsd_surrogate_fallbacks.argtypes = [_P, _I, ctypes.POINTER(_L)]
_lib.mlsd_surrogate_load.argtypes = [_P, ctypes.c_char_p]
_lib.mlsd_surrogate_status.argtypes = [_P, _P]
_lib.mlsd_strerror.argtypes = [_I]
_lib.mlsd_strerror.restype = ctypes.c_char_p


def lib():
    return _lib


def _check(rc, where):
    if rc != 0:
        raise MlsdError(rc, where)


def _dptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Levels:
    """Handle of a built level hierarchy (mlsd_build_levels)."""

    def __init__(self, spectrum, kappa, n_macro, edges, patch_n, patch_div=None, cfl=0.2,
                 t_burn_tau=8.0, t_avg_tau=4.0, n_burn_fixed=0, n_avg_fixed=0,
                 precision="fp32", patch_n_map=None, n_min=0, n_max=0, periodize=False,
                 stream=None):
        k1, k2, re, im = spectrum.as_arrays()
        self._keep = [k1, k2, re, im,
                      np.ascontiguousarray(edges, dtype=np.float64),
                      np.ascontiguousarray(patch_n, dtype=np.int32),
                      None if patch_div is None else np.ascontiguousarray(patch_div, dtype=np.int32)]
        e, pn, pdv = self._keep[4], self._keep[5], self._keep[6]
        nmap = None if patch_n_map is None else np.ascontiguousarray(patch_n_map, dtype=np.int32)
        self._keep.append(nmap)
        self.precision = MLSD_FP64 if precision in ("fp64", MLSD_FP64) else MLSD_FP32
        p = mlsd_problem(n_macro=int(n_macro), kappa=float(kappa), n_modes=len(k1),
                         k1=k1.ctypes.data, k2=k2.ctypes.data, re=re.ctypes.data,
                         im=im.ctypes.data, n_levels=len(e) - 1, band_edges=e.ctypes.data,
                         patch_div=None if pdv is None else pdv.ctypes.data,
                         patch_n=pn.ctypes.data, cfl=float(cfl), t_burn_tau=float(t_burn_tau),
                         t_avg_tau=float(t_avg_tau), n_burn_fixed=int(n_burn_fixed),
                         n_avg_fixed=int(n_avg_fixed), precision=self.precision,
                         patch_n_map=None if nmap is None else nmap.ctypes.data,
                         n_min=int(n_min), n_max=int(n_max), periodize=1 if periodize else 0)
        h = _P()
        _check(_lib.mlsd_build_levels(ctypes.byref(p), _stream(stream), ctypes.byref(h)),
               "mlsd_build_levels")
        self.h = h
        self.n_macro = int(n_macro)
        self.n_levels = len(e) - 1
        self.P = self.n_macro ** 2

    def close(self):
        if getattr(self, "h", None):
            _lib.mlsd_free_levels(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, level):
        d = mlsd_level_desc()
        _check(_lib.mlsd_level_info(self.h, int(level), ctypes.byref(d)), "mlsd_level_info")
        return {f: getattr(d, f) for f, _ in d._fields_}

    def patch_sizes(self, level):
        out = np.zeros(self.P, dtype=np.int32)
        _check(_lib.mlsd_patch_sizes(self.h, int(level), out.ctypes.data), "mlsd_patch_sizes")
        return out

    def features(self, level, B, X, F32=None, stream=None):
        """Surrogate inputs of every patch: X bfloat16 [P][640], F32 [P][606] or None."""
        _check(_lib.mlsd_surrogate_features(self.h, int(level), _dptr(B), _dptr(X), _dptr(F32),
                                            _stream(stream)), "mlsd_surrogate_features")

    def attach_surrogate(self, level, sur, threshold):
        """Use `sur` at `level` in MLSD_SURROGATE chains (None detaches)."""
        self._sur = getattr(self, "_sur", {})
        self._sur[int(level)] = sur                 # keep the handle alive while attached
        _check(_lib.mlsd_attach_surrogate(self.h, int(level), sur.s if sur is not None else None,
                                          float(threshold)), "mlsd_attach_surrogate")

    def surrogate_fallbacks(self, level):
        n = _L()
        _check(_lib.mlsd_surrogate_fallbacks(self.h, int(level), ctypes.byref(n)),
               "mlsd_surrogate_fallbacks")
        return n.value

    def surrogate_dataset(self, level, B, X, Y, stream=None):
        """Plain solves, features X and targets Y of every patch (mlsd_surrogate_dataset)."""
        _check(_lib.mlsd_surrogate_dataset(self.h, int(level), _dptr(B), _dptr(X), _dptr(Y),
                                           _stream(stream)), "mlsd_surrogate_dataset")

    def solve_level_surrogate(self, sur, level, K_base, K_out, threshold, stream=None):
        """Surrogate level solve; returns the number of plain fallback solves."""
        n = _L()
        _check(_lib.mlsd_solve_level_surrogate(self.h, sur.s, int(level), _dptr(K_base),
                                               _dptr(K_out), float(threshold), ctypes.byref(n),
                                               _stream(stream)), "mlsd_solve_level_surrogate")
        return n.value

    def solve_level(self, level, K_base, K_out, w_dump=None, stream=None):
        _check(_lib.mlsd_solve_level(self.h, int(level), _dptr(K_base), _dptr(K_out),
                                     _dptr(w_dump), _stream(stream)), "mlsd_solve_level")

    def offdiag(self, level, B, Koff, stream=None):
        _check(_lib.mlsd_offdiag(self.h, int(level), _dptr(B), _dptr(Koff), _stream(stream)),
               "mlsd_offdiag")

    def effective_diffusivity(self, K_macro, K_levels=None, mode=MLSD_PLAIN, stream=None):
        _check(_lib.mlsd_effective_diffusivity(self.h, int(mode), _dptr(K_macro),
                                               _dptr(K_levels), _stream(stream)),
               "mlsd_effective_diffusivity")

    def status(self, stream=None):
        return _lib.mlsd_status(self.h, _stream(stream))

    def corrector_energy(self, level, K_base, w_dump, E_out, mass_out=None, stream=None):
        """Energy form E (and the means of w) of the correctors in w_dump."""
        _check(_lib.mlsd_corrector_energy(self.h, int(level), _dptr(K_base), _dptr(w_dump),
                                          _dptr(E_out), _dptr(mass_out), _stream(stream)),
               "mlsd_corrector_energy")

    def level_work(self, level, stream=None):
        """(cell-updates, max steps per patch, cell-updates inside the averaging
        window) of the level's last solve."""
        cu, wu, ms = _L(), _L(), _L()
        _check(_lib.mlsd_level_work(self.h, int(level), ctypes.byref(cu), ctypes.byref(wu),
                                    ctypes.byref(ms), _stream(stream)), "mlsd_level_work")
        return cu.value, ms.value, wu.value


    def profile(self, enable=True, serial_classes=False):
        _check(_lib.mlsd_profile(self.h, (2 if serial_classes else 1) if enable else 0),
               "mlsd_profile")

    def profile_collect_classes(self, level, capacity=8):
        """{patch size: (summed patch-kernel ms, launches)} of the level since the last
        collect (size 0: a launch of every size at once)."""
        n = np.zeros(capacity, dtype=np.int32)
        ms = np.zeros(capacity, dtype=np.float64)
        cnt = np.zeros(capacity, dtype=np.int64)
        k = ctypes.c_int32()
        _check(_lib.mlsd_profile_collect_classes(self.h, int(level), capacity, n.ctypes.data,
                                                 ms.ctypes.data, cnt.ctypes.data, ctypes.byref(k)),
               "mlsd_profile_collect_classes")
        return {int(n[i]): (float(ms[i]), int(cnt[i])) for i in range(k.value)}

    def profile_collect(self, level):
        """(summed patch-kernel ms, launches) of the level since the last collect."""
        ms, n = _D(), _L()
        _check(_lib.mlsd_profile_collect(self.h, int(level), ctypes.byref(ms), ctypes.byref(n)),
               "mlsd_profile_collect")
        return ms.value, n.value


def level_schedule(patch_n, patches, schedule):
    """Ticket list [tickets][4] (int64 codes) of the one-launch level kernel for a
    level with the given patch sizes and patch counts (mlsd_level_schedule)."""
    n = np.ascontiguousarray(patch_n, dtype=np.int32)
    c = np.ascontiguousarray(patches, dtype=np.int64)
    nt = _L()
    _lib.mlsd_level_schedule(n.ctypes.data, c.ctypes.data, len(n), int(schedule), 0, None,
                             ctypes.byref(nt))
    if nt.value < 1:
        raise MlsdError(-1, "mlsd_level_schedule")
    out = np.zeros((nt.value, 4), dtype=np.int64)
    _check(_lib.mlsd_level_schedule(n.ctypes.data, c.ctypes.data, len(n), int(schedule),
                                    out.size, out.ctypes.data, ctypes.byref(nt)),
           "mlsd_level_schedule")
    return out


def launch_count():
    return int(_lib.mlsd_launch_count())


def macro_step(U, K, dt, nsteps, want_mass=True, stream=None):
    """In-place Heun steps of U_t = div(K grad U); returns the FP64 mass list."""
    import torch
    prec = MLSD_FP64 if U.dtype == torch.float64 else MLSD_FP32
    mass = np.zeros(nsteps + 1) if want_mass else None
    _check(_lib.mlsd_macro_step(U.shape[0], _dptr(U), prec, _dptr(K), float(dt), int(nsteps),
                                None if mass is None else mass.ctypes.data, _stream(stream)),
           "mlsd_macro_step")
    return mass


def macro_step_dirichlet(U, K, dt, nsteps, u_left=1.0, u_right=0.0, want_mass=False,
                         stream=None):
    """In-place Heun steps with the Sec. 4 boundaries (Dirichlet in x1, periodic
    in x2; column 0 is the boundary x1 = 0); returns the mass list or None."""
    import torch
    prec = MLSD_FP64 if U.dtype == torch.float64 else MLSD_FP32
    mass = np.zeros(nsteps + 1) if want_mass else None
    _check(_lib.mlsd_macro_step_dirichlet(U.shape[0], _dptr(U), prec, _dptr(K), float(dt),
                                          int(nsteps), float(u_left), float(u_right),
                                          None if mass is None else mass.ctypes.data,
                                          _stream(stream)), "mlsd_macro_step_dirichlet")
    return mass


def macro_dt(K, n_macro, cfl, stream=None):
    out = ctypes.c_double()
    _check(_lib.mlsd_macro_dt(int(n_macro), _dptr(K), float(cfl), ctypes.byref(out),
                              _stream(stream)), "mlsd_macro_dt")
    return out.value


def grid_psi(spectrum, nf, psi_out, stream=None):
    k1, k2, re, im = spectrum.as_arrays()
    _check(_lib.mlsd_grid_psi(len(k1), k1.ctypes.data, k2.ctypes.data, re.ctypes.data,
                              im.ctypes.data, int(nf), _dptr(psi_out), _stream(stream)),
           "mlsd_grid_psi")


def dns_run(u, u_tmp, psi, kappa, dt, nsteps, stream=None):
    _check(_lib.mlsd_dns_run(u.shape[0], _dptr(u), _dptr(u_tmp), _dptr(psi), float(kappa),
                             float(dt), int(nsteps), _stream(stream)), "mlsd_dns_run")


def dns_status(stream=None):
    """MLSD_OK, or MLSD_ETIMEOUT if a DNS tile wait ran out since the last call (clears it)."""
    return _lib.mlsd_dns_status(_stream(stream))


def dns_kernel():
    """Name of the DNS kernel this process picked ("" before the first run)."""
    return _lib.mlsd_dns_kernel().decode()


def dns_run_dirichlet(u, u_tmp, psi, kappa, dt, nsteps, u_left=1.0, u_right=0.0, stream=None):
    """Direct simulation with the Sec. 4 boundaries; u, u_tmp float32 or float64, psi float32."""
    import torch
    prec = MLSD_FP64 if u.dtype == torch.float64 else MLSD_FP32
    _check(_lib.mlsd_dns_run_dirichlet(u.shape[0], _dptr(u), _dptr(u_tmp), _dptr(psi), prec,
                                       float(kappa), float(dt), int(nsteps), float(u_left),
                                       float(u_right), _stream(stream)), "mlsd_dns_run_dirichlet")


def dns_dt(psi, kappa, cfl, stream=None):
    out = ctypes.c_double()
    _check(_lib.mlsd_dns_dt(psi.shape[0], _dptr(psi), float(kappa), float(cfl), ctypes.byref(out),
                            _stream(stream)), "mlsd_dns_dt")
    return out.value


def coarse_grain(u, n_macro, U_out, want_mass=True, stream=None):
    m = ctypes.c_double()
    _check(_lib.mlsd_coarse_grain(u.shape[0], _dptr(u), int(n_macro), _dptr(U_out),
                                  ctypes.byref(m) if want_mass else None, _stream(stream)),
           "mlsd_coarse_grain")
    return m.value if want_mass else None


def coarse_grain_noalloc(u, n_macro, U_out, want_mass=True, stream=None):
    """mlsd_coarse_grain_noalloc: same result as coarse_grain, no device allocation."""
    m = ctypes.c_double()
    _check(_lib.mlsd_coarse_grain_noalloc(u.shape[0], _dptr(u), int(n_macro), _dptr(U_out),
                                          ctypes.byref(m) if want_mass else None, _stream(stream)),
           "mlsd_coarse_grain_noalloc")
    return m.value if want_mass else None


def surrogate_symmetry(X, Y, g, X_out, Y_out, stream=None):
    """Images under symmetry g (0..7) of the square of feature rows X (bfloat16
    [n][640]) and targets Y (FP32 [n][3]) into X_out / Y_out (either pair may be
    None) (mlsd_surrogate_symmetry)."""
    n = X.shape[0] if X is not None else Y.shape[0]
    _check(_lib.mlsd_surrogate_symmetry(_dptr(X), _dptr(Y), n, int(g), _dptr(X_out),
                                        _dptr(Y_out), _stream(stream)), "mlsd_surrogate_symmetry")


class Surrogate:
    """Ensemble MLP surrogate handle (mlsd_surrogate_*)."""

    def __init__(self, members=4, hidden=256, max_batch=4096):
        h = _P()
        _check(_lib.mlsd_surrogate_create(int(members), int(hidden), int(max_batch),
                                          ctypes.byref(h)), "mlsd_surrogate_create")
        self.s = h
        self.members, self.hidden, self.max_batch = members, hidden, max_batch
        self.n_params = int(_lib.mlsd_surrogate_param_count(int(hidden)))

    def close(self):
        if getattr(self, "s", None):
            _lib.mlsd_surrogate_free(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, member, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.n_params
        _check(_lib.mlsd_surrogate_set_params(self.s, int(member), p.ctypes.data),
               "mlsd_surrogate_set_params")

    def get_params(self, member):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(_lib.mlsd_surrogate_get_params(self.s, int(member), p.ctypes.data),
               "mlsd_surrogate_get_params")
        return p

    def grad(self, member, X, Y, grad_out=None, stream=None):
        loss = _D()
        _check(_lib.mlsd_surrogate_grad(self.s, int(member), _dptr(X), _dptr(Y), X.shape[0],
                                        _dptr(grad_out), ctypes.byref(loss), _stream(stream)),
               "mlsd_surrogate_grad")
        return loss.value

    def train_step(self, member, X, Y, lr, want_loss=False, stream=None):
        loss = _D()
        _check(_lib.mlsd_surrogate_train_step(self.s, int(member), _dptr(X), _dptr(Y), X.shape[0],
                                              float(lr), ctypes.byref(loss) if want_loss else None,
                                              _stream(stream)), "mlsd_surrogate_train_step")
        return loss.value if want_loss else None

    def train(self, X, Y, epochs, batch, lr, lr_final=None, seed=0, augment=False, stream=None):
        """Adam on every member over the rows of (X, Y) (mlsd_surrogate_train),
        with augment over each row's 8 images under the square's symmetries;
        returns each member's mean loss over the last epoch."""
        losses = np.zeros(self.members)
        lr_final = lr if lr_final is None else lr_final
        _check(_lib.mlsd_surrogate_train(self.s, _dptr(X), _dptr(Y), X.shape[0], int(epochs),
                                         int(batch), float(lr), float(lr_final), int(seed),
                                         1 if augment else 0, losses.ctypes.data,
                                         _stream(stream)), "mlsd_surrogate_train")
        return losses.tolist()

    def save(self, path):
        _check(_lib.mlsd_surrogate_save(self.s, str(path).encode()), "mlsd_surrogate_save")

    def load(self, path):
        _check(_lib.mlsd_surrogate_load(self.s, str(path).encode()), "mlsd_surrogate_load")

    def set_engine(self, engine):
        _check(_lib.mlsd_surrogate_set_engine(self.s, int(engine)), "mlsd_surrogate_set_engine")

    def status(self, stream=None):
        return _lib.mlsd_surrogate_status(self.s, _stream(stream))

    def predict(self, X, out, stream=None):
        _check(_lib.mlsd_surrogate_predict(self.s, _dptr(X), X.shape[0], _dptr(out),
                                           _stream(stream)), "mlsd_surrogate_predict")
