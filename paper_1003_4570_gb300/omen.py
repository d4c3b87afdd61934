"""ctypes binding of libomen.so (argument marshalling only; every step runs in the library).

The functions carry the C names (omen_create, omen_build_lattice, omen_assemble_H, omen_hx,
omen_eigs, ...).  Device buffers are passed as integers (device pointers) or as objects with
a ``data_ptr()`` method (e.g. torch tensors); host buffers as numpy arrays.  A missing or
unloadable library raises immediately: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libomen.so")

OMEN_OK, OMEN_EINVAL, OMEN_ENOMEM, OMEN_ENOCONV, OMEN_ENUMERIC, OMEN_ETIMEOUT, OMEN_ECUDA, OMEN_EUNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ENOCONV", "ENUMERIC", "ETIMEOUT", "ECUDA", "EUNSUPPORTED"]
OMEN_SP3S, OMEN_SP3D5S = 5, 10
OMEN_HARD_WALL, OMEN_PERIODIC, OMEN_BLOCH = 0, 1, 2
OMEN_F64, OMEN_F32, OMEN_F32_REFINE64, OMEN_F64_DF = 0, 1, 2, 3
OMEN_LOWEST, OMEN_NEAREST, OMEN_HIGHEST = 0, 1, 2


class OmenError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("periodic", C.c_int * 3),
                ("a_nm", C.c_double), ("species_host", C.c_void_p), ("strain_host", C.c_void_p)]


class TBParams(C.Structure):
    _fields_ = [("basis", C.c_int), ("nspecies", C.c_int), ("onsite", (C.c_double * 4) * 4),
                ("V", ((C.c_double * 14) * 4) * 4), ("lambda_so", C.c_double * 4), ("eta", C.c_double)]


class HamOpts(C.Structure):
    _fields_ = [("spin_orbit", C.c_int), ("precision", C.c_int), ("matrix_free", C.c_int),
                ("k", C.c_void_p), ("U_atom_dev", C.c_void_p)]


class EigOpts(C.Structure):
    _fields_ = [("nev", C.c_int), ("which", C.c_int), ("sigma", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int), ("block", C.c_int), ("basis", C.c_int), ("v0_host", C.c_void_p),
                ("v0_dev", C.c_void_p)]


class EigInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("hx_count", C.c_longlong), ("restarts", C.c_int),
                ("converged", C.c_int), ("max_residual", C.c_double), ("max_error_bound", C.c_double),
                ("max_residual_raw", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("Lx_nm", C.c_double), ("Ly_nm", C.c_double),
                ("Lz_nm", C.c_double), ("eps_r", C.c_double)]


class CGOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int)]


class TuneResult(C.Structure):
    _fields_ = [("threads", C.c_int), ("rows_per_batch", C.c_int), ("candidates", C.c_int),
                ("ms_best", C.c_double), ("ms_default", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SCFDesc(C.Structure):
    _fields_ = [("lat", C.c_void_p), ("params", C.c_void_p), ("precision", C.c_int), ("grid", C.c_void_p),
                ("donor_rho_dev", C.c_void_p), ("n_electrons", C.c_double), ("kT", C.c_double), ("nk", C.c_int),
                ("k_host", C.c_void_p), ("kw_host", C.c_void_p), ("nev", C.c_int), ("sigma", C.c_double),
                ("e_cut", C.c_double), ("eig_tol", C.c_double), ("eig_block", C.c_int), ("eig_basis", C.c_int),
                ("eig_max_iter", C.c_int), ("mix", C.c_double), ("mix_history", C.c_int), ("tol_V", C.c_double),
                ("max_iter", C.c_int), ("cg", CGOpts), ("poisson_newton", C.c_int)]


class FrozenStates(C.Structure):
    _fields_ = [("nstates", C.c_int), ("E_host", C.c_void_p), ("W_dev", C.c_void_p), ("E_F", C.c_double),
                ("kT", C.c_double), ("phi_in_dev", C.c_void_p)]


class NewtonOpts(C.Structure):
    _fields_ = [("tol_V", C.c_double), ("max_iter", C.c_int), ("cg", CGOpts)]


class NewtonInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("last_step_V", C.c_double),
                ("cg_iterations", C.c_longlong), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SCFInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("dV_inf", C.c_double), ("E_F", C.c_double),
                ("hx_count", C.c_longlong), ("seconds", C.c_double), ("eig_seconds", C.c_double),
                ("poisson_seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EffMassDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h_nm", C.c_double * 3),
                ("m_rel", C.c_double * 3), ("periodic", C.c_int * 3), ("ec_eV", C.c_double),
                ("k", C.c_double * 3), ("precision", C.c_int)]


class VFFParams(C.Structure):
    _fields_ = [("nspecies", C.c_int), ("a_nm", C.c_double * 4), ("alpha", C.c_double * 4), ("beta", C.c_double * 4)]


class VFFOpts(C.Structure):
    _fields_ = [("gtol", C.c_double), ("max_iter", C.c_int)]


class VFFInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("energy_start", C.c_double),
                ("energy", C.c_double), ("max_force", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MLPDesc(C.Structure):
    _fields_ = [("n_in", C.c_int), ("n_hidden1", C.c_int), ("n_hidden2", C.c_int), ("n_out", C.c_int),
                ("feat_log10_shift", C.c_double), ("feat_log10_scale", C.c_double), ("target_scale", C.c_double)]


_lib = None


def lib():
    """Load libomen.so (built in-tree by paper_1003_4570_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        sig = {
            "omen_create": (i, [C.POINTER(vp), i, vp]),
            "omen_destroy": (None, [vp]),
            "omen_last_error": (C.c_char_p, [vp]),
            "omen_set_graph_capture": (i, [vp, i]),
            "omen_set_reorthogonalization": (i, [vp, i]),
            "omen_set_locking_check": (i, [vp, i]),
            "omen_probe_fp64_rate": (i, [vp, C.POINTER(d)]),
            "omen_tune_hx": (i, [vp, vp, i, i, i, C.POINTER(TuneResult)]),
            "omen_tune_hx_kbatch": (i, [vp, vp, i, i, C.POINTER(TuneResult)]),
            "omen_hx_set_tile": (i, [vp, vp, i, i, i]),
            "omen_hx_kbatch_set_tile": (i, [vp, vp, i, i, i]),
            "omen_build_lattice": (i, [vp, C.POINTER(LatticeDesc), C.POINTER(vp)]),
            "omen_free_lattice": (None, [vp]),
            "omen_lattice_counts": (i, [vp, C.POINTER(ll), C.POINTER(ll)]),
            "omen_lattice_set_strain": (i, [vp, vp, vp]),
            "omen_vff_energy_forces": (i, [vp, vp, C.POINTER(VFFParams), vp, vp, C.POINTER(d), vp]),
            "omen_relax_vff": (i, [vp, vp, C.POINTER(VFFParams), vp, C.POINTER(VFFOpts), vp, vp, C.POINTER(VFFInfo)]),
            "omen_assemble_H": (i, [vp, vp, C.POINTER(TBParams), C.POINTER(HamOpts), C.POINTER(vp)]),
            "omen_free_ham": (None, [vp]),
            "omen_assemble_effmass": (i, [vp, C.POINTER(EffMassDesc), vp, C.POINTER(vp)]),
            "omen_ham_shape": (i, [vp, C.POINTER(ll), C.POINTER(i), C.POINTER(i)]),
            "omen_ham_set_potential": (i, [vp, vp, vp]),
            "omen_hx": (i, [vp, vp, vp, vp, i, d]),
            "omen_hx_host": (i, [vp, vp, vp, vp, i, d]),
            "omen_convert_vectors": (i, [vp, vp, i, vp, i, ll]),
            "omen_eigs": (i, [vp, vp, C.POINTER(EigOpts), vp, vp, C.POINTER(EigInfo)]),
            "omen_hx_kbatch": (i, [vp, vp, i, vp, vp, vp, d]),
            "omen_eigs_kbatch": (i, [vp, vp, i, vp, C.POINTER(EigOpts), vp, vp, C.POINTER(EigInfo)]),
            "omen_hx_kbatch_multi": (i, [vp, i, vp, vp, vp, d]),
            "omen_eigs_kbatch_multi": (i, [vp, i, vp, C.POINTER(EigOpts), vp, vp, C.POINTER(EigInfo)]),
            "omen_poisson": (i, [vp, C.POINTER(Grid), vp, vp, C.POINTER(CGOpts), C.POINTER(SolveInfo)]),
            "omen_density_accum": (i, [vp, vp, vp, i, vp, d, vp]),
            "omen_deposit": (i, [vp, vp, C.POINTER(Grid), vp, vp]),
            "omen_gather": (i, [vp, vp, C.POINTER(Grid), vp, vp]),
            "omen_fermi_level": (i, [vp, vp, i, d, d, C.POINTER(d)]),
            "omen_scf": (i, [vp, C.POINTER(SCFDesc), vp, C.POINTER(SCFInfo)]),
            "omen_scf_learned": (i, [vp, C.POINTER(SCFDesc), vp, vp, C.POINTER(SCFInfo), C.POINTER(i)]),
            "omen_poisson_newton": (i, [vp, vp, C.POINTER(Grid), C.POINTER(FrozenStates), vp, vp, C.POINTER(NewtonOpts),
                                        C.POINTER(NewtonInfo)]),
            "omen_state_weights": (i, [vp, vp, vp, i, vp, vp]),
            "omen_mlp_create": (i, [vp, C.POINTER(MLPDesc), vp, C.POINTER(vp)]),
            "omen_mlp_free": (None, [vp]),
            "omen_mlp_param_count": (ll, [vp]),
            "omen_mlp_get_params": (i, [vp, vp, vp, i]),
            "omen_mlp_forward": (i, [vp, vp, vp, i, vp]),
            "omen_mlp_gradients": (i, [vp, vp, vp, vp, i, vp, C.POINTER(C.c_float)]),
            "omen_mlp_train_step": (i, [vp, vp, vp, vp, i, d, C.POINTER(C.c_float)]),
            "omen_mlp_features": (i, [vp, vp, C.POINTER(Grid), vp, vp]),
            "omen_mlp_targets": (i, [vp, vp, C.POINTER(Grid), vp, vp]),
            "omen_mlp_warm_start": (i, [vp, vp, C.POINTER(Grid), vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names the binding expects the library to export."""
    lib()
    return [n for n in dir(_lib) if n.startswith("omen_")]


def _nbytes(buf):
    """Size in bytes of a buffer object (torch tensor or numpy array); None for a raw address."""
    if buf is None or isinstance(buf, int):
        return None
    if hasattr(buf, "numel") and hasattr(buf, "element_size"):
        return int(buf.numel()) * int(buf.element_size())
    if isinstance(buf, np.ndarray):
        return int(buf.nbytes)
    return None


def _need(buf, nbytes, what):
    """Refuse a buffer smaller than what the library will read or write through it."""
    have = _nbytes(buf)
    if have is not None and have < nbytes:
        raise ValueError(f"{what}: buffer of {have} bytes, the call uses {nbytes}")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


class Context:
    def __init__(self, handle):
        self.handle = handle

    def check(self, status):
        if status != OMEN_OK:
            raise OmenError(status, lib().omen_last_error(self.handle).decode())
        return status

    def close(self):
        if self.handle:
            lib().omen_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def omen_create(device=0, stream=None) -> Context:
    h = C.c_void_p()
    s = lib().omen_create(C.byref(h), int(device), _ptr(stream) if stream is not None else None)
    if s != OMEN_OK:
        raise OmenError(s, "omen_create failed (no CUDA device?)")
    return Context(h)


OMEN_REORTH_FULL, OMEN_REORTH_SEMI, OMEN_REORTH_PARTIAL = 0, 1, 2


def omen_set_reorthogonalization(ctx: Context, policy) -> None:
    ctx.check(lib().omen_set_reorthogonalization(ctx.handle, int(policy)))


def omen_probe_fp64_rate(ctx: Context) -> float:
    """Measured FP64 FMA rate of the device (TFLOP/s)."""
    t = C.c_double()
    ctx.check(lib().omen_probe_fp64_rate(ctx.handle, C.byref(t)))
    return t.value


def omen_set_locking_check(ctx: Context, enable: bool) -> None:
    ctx.check(lib().omen_set_locking_check(ctx.handle, int(bool(enable))))


def omen_set_graph_capture(ctx: Context, enable: bool) -> None:
    ctx.check(lib().omen_set_graph_capture(ctx.handle, int(bool(enable))))


class Lattice:
    def __init__(self, ctx, handle, keep):
        self.ctx, self.handle, self._keep = ctx, handle, keep

    def counts(self):
        n, b = C.c_longlong(), C.c_longlong()
        lib().omen_lattice_counts(self.handle, C.byref(n), C.byref(b))
        return n.value, b.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib().omen_free_lattice(self.handle)
            self.handle = None


def omen_build_lattice(ctx: Context, spec) -> Lattice:
    """spec: nx, ny, nz, periodic (3), a_nm, species (uint8[8*ncells]), strain (float64[16*ncells])."""
    species = np.ascontiguousarray(spec.species, dtype=np.uint8)
    strain = None if spec.strain is None else np.ascontiguousarray(spec.strain, dtype=np.float64)
    d = LatticeDesc(spec.nx, spec.ny, spec.nz, (C.c_int * 3)(*spec.periodic), float(spec.a_nm),
                    species.ctypes.data, None if strain is None else strain.ctypes.data)
    h = C.c_void_p()
    ctx.check(lib().omen_build_lattice(ctx.handle, C.byref(d), C.byref(h)))
    return Lattice(ctx, h, (species, strain))


def omen_lattice_set_strain(ctx: Context, lat: Lattice, strain_dev) -> None:
    """Replace the structure's per-slot bond strains (device, [16*ncells] float64)."""
    natoms, _ = lat.counts()
    _need(strain_dev, 16 * (natoms // 8) * 8, "strain_dev")
    ctx.check(lib().omen_lattice_set_strain(ctx.handle, lat.handle, _ptr(strain_dev)))


def vff_params_struct(vp) -> VFFParams:
    """vp: a_nm, alpha, beta per species (arrays of equal length <= 4; eV/nm^2 for alpha, beta)."""
    a = np.asarray(vp.a_nm, dtype=np.float64).ravel()
    t = VFFParams()
    t.nspecies = len(a)
    for q in range(len(a)):
        t.a_nm[q] = float(a[q])
        t.alpha[q] = float(np.asarray(vp.alpha).ravel()[q])
        t.beta[q] = float(np.asarray(vp.beta).ravel()[q])
    return t


def _box(F):
    if F is None:
        return None
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(3, 3)
    return F


def omen_vff_energy_forces(ctx: Context, lat: Lattice, vp, u_dev, F=None, force_dev=None):
    """Keating energy (eV) at displacements u_dev ([3][natoms] float64, nm); forces -dE/du into
    force_dev ([3][natoms]) when given."""
    natoms, _ = lat.counts()
    _need(u_dev, 3 * natoms * 8, "u_dev")
    if force_dev is not None:
        _need(force_dev, 3 * natoms * 8, "force_dev")
    t = vff_params_struct(vp)
    Fb = _box(F)
    E = C.c_double()
    ctx.check(lib().omen_vff_energy_forces(ctx.handle, lat.handle, C.byref(t), None if Fb is None else Fb.ctypes.data,
                                           _ptr(u_dev), C.byref(E), _ptr(force_dev)))
    return E.value


def omen_relax_vff(ctx: Context, lat: Lattice, vp, u_dev, F=None, gtol=1e-10, max_iter=20000, strain_dev=None,
                   raise_on_noconv=True):
    """Relax u_dev in place at box deformation F; relaxed bond strains into strain_dev ([16*ncells])
    when given.  Returns (info dict, status)."""
    natoms, _ = lat.counts()
    _need(u_dev, 3 * natoms * 8, "u_dev")
    if strain_dev is not None:
        _need(strain_dev, 16 * (natoms // 8) * 8, "strain_dev")
    t = vff_params_struct(vp)
    Fb = _box(F)
    o = VFFOpts(float(gtol), int(max_iter))
    info = VFFInfo()
    s = lib().omen_relax_vff(ctx.handle, lat.handle, C.byref(t), None if Fb is None else Fb.ctypes.data, C.byref(o),
                             _ptr(u_dev), _ptr(strain_dev), C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    return info.as_dict(), s


def tb_params_struct(p) -> TBParams:
    """p: basis, onsite (ns,4), V (ns,ns,14), lambda_so (ns,), eta."""
    t = TBParams()
    ns = p.onsite.shape[0]
    t.basis, t.nspecies, t.eta = int(p.basis), ns, float(p.eta)
    for a in range(ns):
        for q in range(4):
            t.onsite[a][q] = float(p.onsite[a, q])
        t.lambda_so[a] = float(p.lambda_so[a])
        for b in range(ns):
            for q in range(14):
                t.V[a][b][q] = float(p.V[a, b, q])
    return t


class Hamiltonian:
    def __init__(self, ctx, handle, lat, precision=OMEN_F64):
        self.ctx, self.handle, self.lattice = ctx, handle, lat
        self.precision = int(precision)
        n, c, e = C.c_longlong(), C.c_int(), C.c_int()
        lib().omen_ham_shape(handle, C.byref(n), C.byref(c), C.byref(e))
        self.nrows, self.is_complex, self.elem_bytes = n.value, bool(c.value), e.value

    @property
    def evec_bytes(self):
        """Bytes per element of the eigenvectors omen_eigs returns: FP64 (complex128) except for
        OMEN_F32 Hamiltonians, whose eigenvectors are in their own vector type."""
        if self.precision == OMEN_F32:
            return self.elem_bytes
        return 16 if self.is_complex else 8

    @property
    def numpy_dtype(self):
        """dtype of host vectors (omen_hx_host); double-float Hamiltonians take FP64 on the host."""
        if self.is_complex:
            return np.complex128 if self.elem_bytes == 16 else np.complex64
        return np.float64 if self.elem_bytes == 8 else np.float32

    def __del__(self):
        if getattr(self, "handle", None):
            lib().omen_free_ham(self.handle)
            self.handle = None


def omen_assemble_H(ctx: Context, lat: Lattice, params, spin_orbit=False, precision=OMEN_F64,
                    matrix_free=False, k=None, U_atom_dev=None) -> Hamiltonian:
    tp = tb_params_struct(params)
    karr = None if k is None else np.ascontiguousarray(k, dtype=np.float64)
    o = HamOpts(int(bool(spin_orbit)), int(precision), int(bool(matrix_free)),
                None if karr is None else karr.ctypes.data, _ptr(U_atom_dev))
    h = C.c_void_p()
    ctx.check(lib().omen_assemble_H(ctx.handle, lat.handle, C.byref(tp), C.byref(o), C.byref(h)))
    return Hamiltonian(ctx, h, lat, precision)


def omen_assemble_effmass(ctx: Context, spec, precision=OMEN_F64, U_dev=None) -> Hamiltonian:
    """Single-band effective-mass Hamiltonian on a uniform grid.  spec: nx, ny, nz, h_nm[3],
    m_rel[3], periodic[3], ec_eV, kvec ([3] 1/nm or None); U_dev: device potential per point."""
    d = EffMassDesc()
    d.nx, d.ny, d.nz = int(spec.nx), int(spec.ny), int(spec.nz)
    kv = (0.0, 0.0, 0.0) if spec.kvec is None else spec.kvec
    for a in range(3):
        d.h_nm[a] = float(spec.h_nm[a])
        d.m_rel[a] = float(spec.m_rel[a])
        d.periodic[a] = int(spec.periodic[a])
        d.k[a] = float(kv[a])
    d.ec_eV = float(spec.ec_eV)
    d.precision = int(precision)
    h = C.c_void_p()
    ctx.check(lib().omen_assemble_effmass(ctx.handle, C.byref(d), _ptr(U_dev), C.byref(h)))
    return Hamiltonian(ctx, h, None, precision)


def omen_ham_set_potential(ctx: Context, ham: Hamiltonian, U_atom_dev):
    ctx.check(lib().omen_ham_set_potential(ctx.handle, ham.handle, _ptr(U_atom_dev)))


def omen_hx(ctx: Context, ham: Hamiltonian, x_dev, y_dev, nvec=1, sigma=0.0):
    """y = (H - sigma) x on device buffers (asynchronous on the context's stream)."""
    _need(x_dev, int(nvec) * ham.nrows * ham.elem_bytes, "omen_hx x")
    _need(y_dev, int(nvec) * ham.nrows * ham.elem_bytes, "omen_hx y")
    ctx.check(lib().omen_hx(ctx.handle, ham.handle, _ptr(x_dev), _ptr(y_dev), int(nvec), float(sigma)))


def omen_hx_host(ctx: Context, ham: Hamiltonian, x: np.ndarray, sigma=0.0) -> np.ndarray:
    """The same product on host arrays of shape (nvec, nrows) or (nrows,)."""
    x = np.ascontiguousarray(x, dtype=ham.numpy_dtype)
    nvec = 1 if x.ndim == 1 else x.shape[0]
    y = np.empty_like(x)
    ctx.check(lib().omen_hx_host(ctx.handle, ham.handle, x.ctypes.data, y.ctypes.data, nvec, float(sigma)))
    return y


def omen_eigs(ctx: Context, ham: Hamiltonian, nev, which=OMEN_LOWEST, sigma=0.0, tol=1e-9, max_iter=1000,
              block=1, basis=None, v0=None, evecs_dev=None, raise_on_noconv=True, v0_dev=None):
    """Eigenpairs by thick-restart block Lanczos.  Returns (evals ndarray, info dict, status)."""
    _need(evecs_dev, int(nev) * ham.nrows * ham.evec_bytes, "omen_eigs evecs")
    _need(v0_dev, int(block) * ham.nrows * ham.elem_bytes, "omen_eigs v0")
    if basis is None:
        basis = max(4 * block, ((2 * nev + 2 * block + block - 1) // block) * block, 32 // block * block)
    v0a = None
    if v0 is not None:
        v0a = np.ascontiguousarray(v0, dtype=ham.numpy_dtype)
    o = EigOpts(int(nev), int(which), float(sigma), float(tol), int(max_iter), int(block), int(basis),
                None if v0a is None else v0a.ctypes.data, _ptr(v0_dev))
    ev = np.zeros(nev)
    info = EigInfo()
    s = lib().omen_eigs(ctx.handle, ham.handle, C.byref(o), ev.ctypes.data, _ptr(evecs_dev), C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    return ev, info.as_dict(), s


def grid_struct(g) -> Grid:
    """g: nx, ny, nz, Lx_nm, Ly_nm, Lz_nm, eps_r (e.g. oracle.poisson.Grid or any namespace)."""
    return Grid(int(g.nx), int(g.ny), int(g.nz), float(g.Lx_nm), float(g.Ly_nm), float(g.Lz_nm), float(g.eps_r))


def omen_poisson(ctx: Context, grid, rho_dev, phi_dev, rtol=1e-12, max_iter=100000, precision=OMEN_F64):
    """CG solve in place on phi_dev (initial guess in).  precision OMEN_F64, or OMEN_F32_REFINE64
    for FP32 iterations with FP64 residual replacement.  Returns the solve info dict."""
    g = grid_struct(grid)
    o = CGOpts(float(rtol), int(max_iter), int(precision))
    info = SolveInfo()
    ctx.check(lib().omen_poisson(ctx.handle, C.byref(g), _ptr(rho_dev), _ptr(phi_dev), C.byref(o), C.byref(info)))
    return info.as_dict()


def omen_density_accum(ctx: Context, ham: Hamiltonian, psi_dev, nstates, occ, weight, n_atom_dev):
    _need(psi_dev, int(nstates) * ham.nrows * (16 if ham.is_complex else 8), "omen_density_accum psi")
    occ = np.ascontiguousarray(occ, dtype=np.float64)
    ctx.check(lib().omen_density_accum(ctx.handle, ham.handle, _ptr(psi_dev), int(nstates), occ.ctypes.data,
                                       float(weight), _ptr(n_atom_dev)))


def omen_deposit(ctx: Context, lat: Lattice, grid, q_atom_dev, rho_dev):
    g = grid_struct(grid)
    ctx.check(lib().omen_deposit(ctx.handle, lat.handle, C.byref(g), _ptr(q_atom_dev), _ptr(rho_dev)))


def omen_gather(ctx: Context, lat: Lattice, grid, phi_dev, phi_atom_dev):
    g = grid_struct(grid)
    ctx.check(lib().omen_gather(ctx.handle, lat.handle, C.byref(g), _ptr(phi_dev), _ptr(phi_atom_dev)))


def omen_fermi_level(E, level_weight, n_target, kT):
    E = np.ascontiguousarray(E, dtype=np.float64)
    w = np.ascontiguousarray(level_weight, dtype=np.float64)
    ef = C.c_double()
    s = lib().omen_fermi_level(E.ctypes.data, w.ctypes.data, len(E), float(n_target), float(kT), C.byref(ef))
    if s != OMEN_OK:
        raise OmenError(s, "omen_fermi_level: target not reachable or bad arguments")
    return ef.value


def omen_scf(ctx: Context, lat: Lattice, params, grid, phi_dev, donor_rho_dev, n_electrons, kT, kpts, kweights,
             nev, sigma, e_cut, precision=OMEN_F64, eig_tol=1e-9, eig_block=1, eig_basis=None, eig_max_iter=20000,
             mix=0.1, tol_V=1e-6, max_iter=300, cg_rtol=1e-13, cg_max_iter=100000, raise_on_noconv=True,
             mix_history=0, poisson_newton=False):
    """Self-consistent loop in place on phi_dev.  Returns (info dict, status)."""
    tp = tb_params_struct(params)
    g = grid_struct(grid)
    k = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    kw = np.ascontiguousarray(kweights, dtype=np.float64)
    if eig_basis is None:
        eig_basis = max(4 * eig_block, ((2 * nev + 2 * eig_block + eig_block - 1) // eig_block) * eig_block)
    d = SCFDesc(lat.handle, C.addressof(tp), int(precision), C.addressof(g), _ptr(donor_rho_dev), float(n_electrons),
                float(kT), len(kw), k.ctypes.data, kw.ctypes.data, int(nev), float(sigma), float(e_cut), float(eig_tol),
                int(eig_block), int(eig_basis), int(eig_max_iter), float(mix), int(mix_history), float(tol_V),
                int(max_iter), CGOpts(float(cg_rtol), int(cg_max_iter)), int(bool(poisson_newton)))
    info = SCFInfo()
    s = lib().omen_scf(ctx.handle, C.byref(d), _ptr(phi_dev), C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    return info.as_dict(), s


def omen_state_weights(ctx: Context, ham: Hamiltonian, psi_dev, nstates, weights, W_dev) -> None:
    """W_dev[n][atom] = weights[n] * sum_orb |psi_n|^2 (FP64 eigenvectors of a tight-binding H)."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    natoms, _ = ham.lattice.counts()
    _need(psi_dev, int(nstates) * ham.nrows * ham.evec_bytes, "psi_dev")
    _need(W_dev, int(nstates) * natoms * 8, "W_dev")
    ctx.check(lib().omen_state_weights(ctx.handle, ham.handle, _ptr(psi_dev), int(nstates), w.ctypes.data, _ptr(W_dev)))


def omen_poisson_newton(ctx: Context, lat: Lattice, grid, E, W_dev, E_F, kT, phi_in_dev, rho_d_dev, phi_dev,
                        tol_V=1e-10, max_iter=50, cg_rtol=1e-12, cg_max_iter=100000, raise_on_noconv=True):
    """Root of the nonlinear Poisson equation with the frozen states' predicted charge, in place
    on phi_dev.  Returns (info dict, status)."""
    g = grid_struct(grid)
    E = np.ascontiguousarray(E, dtype=np.float64)
    fs = FrozenStates(len(E), E.ctypes.data if len(E) else None, _ptr(W_dev), float(E_F), float(kT), _ptr(phi_in_dev))
    o = NewtonOpts(float(tol_V), int(max_iter), CGOpts(float(cg_rtol), int(cg_max_iter)))
    info = NewtonInfo()
    s = lib().omen_poisson_newton(ctx.handle, lat.handle, C.byref(g), C.byref(fs), _ptr(rho_d_dev), _ptr(phi_dev),
                                  C.byref(o), C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    return info.as_dict(), s


def _scf_desc(lat, params, grid, donor_rho_dev, n_electrons, kT, kpts, kweights, nev, sigma, e_cut, precision,
              eig_tol, eig_block, eig_basis, eig_max_iter, mix, tol_V, max_iter, cg_rtol, cg_max_iter, mix_history,
              poisson_newton):
    tp = tb_params_struct(params)
    g = grid_struct(grid)
    k = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    kw = np.ascontiguousarray(kweights, dtype=np.float64)
    if eig_basis is None:
        eig_basis = max(4 * eig_block, ((2 * nev + 2 * eig_block + eig_block - 1) // eig_block) * eig_block)
    d = SCFDesc(lat.handle, C.addressof(tp), int(precision), C.addressof(g), _ptr(donor_rho_dev), float(n_electrons),
                float(kT), len(kw), k.ctypes.data, kw.ctypes.data, int(nev), float(sigma), float(e_cut), float(eig_tol),
                int(eig_block), int(eig_basis), int(eig_max_iter), float(mix), int(mix_history), float(tol_V),
                int(max_iter), CGOpts(float(cg_rtol), int(cg_max_iter)), int(bool(poisson_newton)))
    return d, (tp, g, k, kw)


def omen_scf_learned(ctx: Context, mlp, lat: Lattice, params, grid, phi_dev, donor_rho_dev, n_electrons, kT, kpts,
                     kweights, nev, sigma, e_cut, precision=OMEN_F64, eig_tol=1e-9, eig_block=1, eig_basis=None,
                     eig_max_iter=20000, mix=0.1, tol_V=1e-6, max_iter=300, cg_rtol=1e-13, cg_max_iter=100000,
                     mix_history=0, poisson_newton=False):
    """omen_scf from the network's start, falling back to zero field.  Returns (info, status, fallback)."""
    d, keep = _scf_desc(lat, params, grid, donor_rho_dev, n_electrons, kT, kpts, kweights, nev, sigma, e_cut,
                        precision, eig_tol, eig_block, eig_basis, eig_max_iter, mix, tol_V, max_iter, cg_rtol,
                        cg_max_iter, mix_history, poisson_newton)
    info = SCFInfo()
    fb = C.c_int()
    s = lib().omen_scf_learned(ctx.handle, C.byref(d), mlp.handle, _ptr(phi_dev), C.byref(info), C.byref(fb))
    ctx.check(s)
    return info.as_dict(), s, bool(fb.value)


def omen_tune_hx(ctx: Context, ham: Hamiltonian, vec_precision=None, nvec=1, reps=10) -> dict:
    """Time the compiled launch shapes of the product on this Hamiltonian; keep the fastest."""
    if vec_precision is None:
        vec_precision = OMEN_F32 if ham.elem_bytes == (8 if ham.is_complex else 4) else OMEN_F64
    r = TuneResult()
    ctx.check(lib().omen_tune_hx(ctx.handle, ham.handle, int(vec_precision), int(nvec), int(reps), C.byref(r)))
    return r.as_dict()


def omen_tune_hx_kbatch(ctx: Context, ham: Hamiltonian, nk, reps=10) -> dict:
    r = TuneResult()
    ctx.check(lib().omen_tune_hx_kbatch(ctx.handle, ham.handle, int(nk), int(reps), C.byref(r)))
    return r.as_dict()


def omen_hx_set_tile(ctx: Context, ham: Hamiltonian, vec_precision, threads, rows_per_batch) -> None:
    ctx.check(lib().omen_hx_set_tile(ctx.handle, ham.handle, int(vec_precision), int(threads), int(rows_per_batch)))


def omen_hx_kbatch_set_tile(ctx: Context, ham: Hamiltonian, vec_precision, threads, k_per_thread) -> None:
    ctx.check(lib().omen_hx_kbatch_set_tile(ctx.handle, ham.handle, int(vec_precision), int(threads), int(k_per_thread)))


def omen_hx_kbatch(ctx: Context, ham: Hamiltonian, kpts, x_dev, y_dev, sigma=0.0):
    """y_k = (H(k) - sigma) x_k for every wave vector (device buffers [nk][nrows])."""
    k = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    _need(x_dev, len(k) * ham.nrows * ham.elem_bytes, "omen_hx_kbatch x")
    _need(y_dev, len(k) * ham.nrows * ham.elem_bytes, "omen_hx_kbatch y")
    ctx.check(lib().omen_hx_kbatch(ctx.handle, ham.handle, len(k), k.ctypes.data, _ptr(x_dev), _ptr(y_dev), float(sigma)))


def omen_eigs_kbatch(ctx: Context, ham: Hamiltonian, kpts, nev, which=OMEN_LOWEST, sigma=0.0, tol=1e-9,
                     max_iter=1000, basis=None, evecs_dev=None, raise_on_noconv=True):
    """nev eigenpairs per wave vector, all k in lockstep.  Returns (evals [nk, nev], info, status)."""
    k = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    if basis is None:
        basis = max(32, 2 * nev + 4)
    o = EigOpts(int(nev), int(which), float(sigma), float(tol), int(max_iter), 1, int(basis), None, None)
    ev = np.zeros((len(k), nev))
    info = EigInfo()
    s = lib().omen_eigs_kbatch(ctx.handle, ham.handle, len(k), k.ctypes.data, C.byref(o), ev.ctypes.data,
                               _ptr(evecs_dev), C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    return ev, info.as_dict(), s


class KbatchItem(C.Structure):
    _fields_ = [("ham", C.c_void_p), ("nk", C.c_int), ("k_host", C.c_void_p)]


def _kbatch_items(items):
    """items: sequence of (Hamiltonian, wave vectors [nk, 3]) -> ctypes array and kept arrays."""
    ks = [np.ascontiguousarray(k, dtype=np.float64).reshape(-1, 3) for _, k in items]
    arr = (KbatchItem * len(items))(*[KbatchItem(h.handle, len(k), k.ctypes.data) for (h, _), k in zip(items, ks)])
    return arr, ks


def omen_hx_kbatch_multi(ctx: Context, items, x_dev, y_dev, sigma=0.0):
    """One launch over every (structure, k): vectors of the items one after another."""
    arr, keep = _kbatch_items(items)
    ctx.check(lib().omen_hx_kbatch_multi(ctx.handle, len(items), arr, _ptr(x_dev), _ptr(y_dev), float(sigma)))


def omen_eigs_kbatch_multi(ctx: Context, items, nev, which=OMEN_LOWEST, sigma=0.0, tol=1e-9, max_iter=1000,
                           basis=None, evecs_dev=None, raise_on_noconv=True):
    """Lockstep solve over several structures.  Returns ([evals [nk_i, nev] per item], info, status)."""
    arr, ks = _kbatch_items(items)
    if basis is None:
        basis = max(32, 2 * nev + 4)
    o = EigOpts(int(nev), int(which), float(sigma), float(tol), int(max_iter), 1, int(basis), None, None)
    total = sum(len(k) for k in ks)
    ev = np.zeros((total, nev))
    info = EigInfo()
    s = lib().omen_eigs_kbatch_multi(ctx.handle, len(items), arr, C.byref(o), ev.ctypes.data, _ptr(evecs_dev),
                                     C.byref(info))
    if s != OMEN_OK and not (s == OMEN_ENOCONV and not raise_on_noconv):
        ctx.check(s)
    out, i0 = [], 0
    for k in ks:
        out.append(ev[i0:i0 + len(k)])
        i0 += len(k)
    return out, info.as_dict(), s


class MLP:
    def __init__(self, ctx, handle, desc):
        self.ctx, self.handle, self.desc = ctx, handle, desc

    @property
    def nparams(self):
        return lib().omen_mlp_param_count(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            lib().omen_mlp_free(self.handle)
            self.handle = None


def omen_mlp_create(ctx: Context, params, sizes=(256, 512, 512, 256), feat_shift=21.0, feat_scale=6.0,
                    target_scale=0.2) -> MLP:
    p = np.ascontiguousarray(params, dtype=np.float32)
    d = MLPDesc(*[int(v) for v in sizes], float(feat_shift), float(feat_scale), float(target_scale))
    h = C.c_void_p()
    ctx.check(lib().omen_mlp_create(ctx.handle, C.byref(d), p.ctypes.data, C.byref(h)))
    return MLP(ctx, h, d)


def omen_mlp_get_params(ctx: Context, mlp: MLP, bf16_rounded=False):
    out = np.zeros(mlp.nparams, np.float32)
    ctx.check(lib().omen_mlp_get_params(ctx.handle, mlp.handle, out.ctypes.data, int(bool(bf16_rounded))))
    return out


def omen_mlp_forward(ctx: Context, mlp: MLP, X_dev, batch, Y_dev):
    ctx.check(lib().omen_mlp_forward(ctx.handle, mlp.handle, _ptr(X_dev), int(batch), _ptr(Y_dev)))


def omen_mlp_gradients(ctx: Context, mlp: MLP, X_dev, T_dev, batch):
    g = np.zeros(mlp.nparams, np.float32)
    loss = C.c_float()
    ctx.check(lib().omen_mlp_gradients(ctx.handle, mlp.handle, _ptr(X_dev), _ptr(T_dev), int(batch), g.ctypes.data,
                                       C.byref(loss)))
    return g, loss.value


def omen_mlp_train_step(ctx: Context, mlp: MLP, X_dev, T_dev, batch, lr=1e-3, want_loss=True):
    loss = C.c_float()
    ctx.check(lib().omen_mlp_train_step(ctx.handle, mlp.handle, _ptr(X_dev), _ptr(T_dev), int(batch), float(lr),
                                        C.byref(loss) if want_loss else None))
    return loss.value


def omen_mlp_features(ctx: Context, mlp: MLP, grid, donor_rho_dev, x_dev):
    g = grid_struct(grid)
    ctx.check(lib().omen_mlp_features(ctx.handle, mlp.handle, C.byref(g), _ptr(donor_rho_dev), _ptr(x_dev)))


def omen_mlp_targets(ctx: Context, mlp: MLP, grid, phi_dev, t_dev):
    g = grid_struct(grid)
    ctx.check(lib().omen_mlp_targets(ctx.handle, mlp.handle, C.byref(g), _ptr(phi_dev), _ptr(t_dev)))


def omen_mlp_warm_start(ctx: Context, mlp: MLP, grid, donor_rho_dev, phi_dev):
    g = grid_struct(grid)
    ctx.check(lib().omen_mlp_warm_start(ctx.handle, mlp.handle, C.byref(g), _ptr(donor_rho_dev), _ptr(phi_dev)))
