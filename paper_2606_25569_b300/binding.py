"""Thin ctypes binding of the vesb300 C ABI (include/vesb300.h): argument marshalling only.

Every computation runs in libvesb300.so. Loading fails loudly when the library is missing;
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvesb300.so")

VS_FLAG_FARFIELD_FP64 = 1
VS_FLAG_DIRECT_FP64 = 2
VS_FLAG_NO_AUTOTUNE = 4
VS_FLAG_TC_GEMM = 8
VS_FLAG_FARFIELD_MULTIPOLE = 16
VS_FLAG_FARFIELD_PER_TARGET = 32
VS_FLAG_NEAR_YZ = 64
VS_FLAG_OPS_BATCHED = 128
VS_FLAG_FARFIELD_TREE = 256

STATUS = {0: "VS_OK", 1: "VS_ERR_INVALID_ARG", 2: "VS_ERR_CUDA", 3: "VS_ERR_NOMEM",
          4: "VS_ERR_NOT_CONVERGED", 5: "VS_ERR_UNSTABLE", 6: "VS_ERR_TIMEOUT", 7: "VS_ERR_NO_NETWORK"}

FUNCTIONS = {
    "vs_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "vs_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "vs_set_near_networks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32]),
    "vs_near_maps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "vs_set_gmres": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int32]),
    "vs_gmres_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_get_positions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_get_tension": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_get_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_get_reference": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_get_device_ptrs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_get_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_get_hybrid_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "vs_farfield_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "vs_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "vs_set_network": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_int32]),
    "vs_relax": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_set_flow_networks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32]),
    "vs_flow_maps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "vs_training_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_int32]),
    "vs_checkpoint_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_checkpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_restore": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vs_destroy": (None, [ctypes.c_void_p]),
    "vs_farfield_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_farfield_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_farfield_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_farfield_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vs_farfield_plan_destroy": (None, [ctypes.c_void_p]),
    "vs_farfield_eval_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_batched_inverse32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "vs_fp32_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_mlp_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "vs_mlp_num_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_mlp_set_affine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "vs_mlp_get_affine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "vs_mlp_fit_affine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_double]),
    "vs_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "vs_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "vs_mlp_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "vs_mlp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vs_mlp_destroy": (None, [ctypes.c_void_p]),
    "vs_ivnet_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_ivnet_num_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vs_ivnet_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_ivnet_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_ivnet_set_affine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "vs_ivnet_fit_affine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_double]),
    "vs_ivnet_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "vs_ivnet_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "vs_ivnet_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "vs_ivnet_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "vs_ivnet_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vs_ivnet_destroy": (None, [ctypes.c_void_p]),
    "vs_feature_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_standardize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vs_self_matrices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]),
}

_lib = None


def lib():
    """Load libvesb300.so (built in-tree by paper_2606_25569_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libvesb300.so is not built: run python -m paper_2606_25569_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in FUNCTIONS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class VsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class VsParams(ctypes.Structure):
    _fields_ = [("kappa_b", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
                ("corr_tol", ctypes.c_double), ("mode", ctypes.c_int32), ("near_field", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("exact_every", ctypes.c_int32), ("flags", ctypes.c_uint64),
                ("exact_gap", ctypes.c_double)]


class VsFlow(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32), ("p", ctypes.c_double * 4)]


def _ptr(a):
    """Device/host address of a numpy array or a torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    return int(a)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Suspension:
    """Owner of a vs_suspension handle (vs_create ... vs_destroy)."""

    def __init__(self, xy, offsets, kappa=1.0, mu=1.0, dt=1e-4, corr_tol=0.01, flow_kind=0,
                 flow_p=(0.0, 0.0, 0.0, 0.0), near_field=False, farfield_fp64=False, stream=None, mode=0,
                 use_graph=False, direct_fp64=False, autotune=True, tc_gemm=False, exact_every=0,
                 farfield_multipole=False, farfield_per_target=False, exact_gap=0.0, near_yz=False,
                 farfield_tree=False,
                 ops_batched=False):
        L = lib()
        self._h = ctypes.c_void_p()
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self.M = len(off) - 1
        self.P = int(off[-1])
        flags = ((VS_FLAG_FARFIELD_FP64 if farfield_fp64 else 0) | (VS_FLAG_DIRECT_FP64 if direct_fp64 else 0)
                 | (0 if autotune else VS_FLAG_NO_AUTOTUNE) | (VS_FLAG_TC_GEMM if tc_gemm else 0)
                 | (VS_FLAG_FARFIELD_MULTIPOLE if farfield_multipole else 0)
                 | (VS_FLAG_FARFIELD_TREE if farfield_tree else 0)
                 | (VS_FLAG_FARFIELD_PER_TARGET if farfield_per_target else 0)
                 | (VS_FLAG_NEAR_YZ if near_yz else 0) | (VS_FLAG_OPS_BATCHED if ops_batched else 0))
        p = VsParams(kappa, mu, dt, corr_tol, int(mode), 1 if near_field else 0, 1 if use_graph else 0,
                     int(exact_every), flags, float(exact_gap))
        f = VsFlow(int(flow_kind), 0, (ctypes.c_double * 4)(*[float(v) for v in flow_p]))
        st = L.vs_create(_ptr(xy), _ptr(off), self.M, ctypes.byref(p), ctypes.byref(f), _stream(stream),
                         ctypes.byref(self._h))
        if st != 0:
            raise VsError(st, L.vs_last_error(None).decode())

    def _check(self, st):
        if st != 0:
            raise VsError(st, lib().vs_last_error(self._h).decode())

    def step(self, n=1):
        self._check(lib().vs_step(self._h, int(n)))

    def sync(self):
        self._check(lib().vs_sync(self._h))

    def set_state(self, xy, sigma):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        self._check(lib().vs_set_state(self._h, _ptr(xy), _ptr(sigma)))

    def _get(self, fn, n):
        out = np.empty(n)
        self._check(fn(self._h, _ptr(out), n))
        return out

    def positions(self):
        return self._get(lib().vs_get_positions, 2 * self.P)

    def tension(self):
        return self._get(lib().vs_get_tension, self.P)

    def velocity(self):
        return self._get(lib().vs_get_velocity, 2 * self.P)

    def reference(self):
        r = self._get(lib().vs_get_reference, 2 * self.M)
        return r[:self.M], r[self.M:]

    def farfield_variant(self, set=-1):
        """(index, threads per CTA, staged points) of the FP32 far field in use (index -1: the symmetric
        kernel); set >= 0 selects a per-target launch shape."""
        idx, thr, chk = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().vs_farfield_variant(self._h, int(set), ctypes.byref(idx), ctypes.byref(thr),
                                              ctypes.byref(chk)))
        return idx.value, thr.value, chk.value

    def counters(self):
        out = np.zeros(5, dtype=np.int64)
        self._check(lib().vs_get_counters(self._h, _ptr(out)))
        return {"steps": int(out[0]), "corrections": int(out[1]), "near_pairs": int(out[2]), "err": int(out[3]),
                "launches": int(out[4])}

    def hybrid_counters(self):
        """Hybrid fallback statistics: learned relaxation steps, steps with the fallback test, and vesicles
        stepped exactly in them (summed over those steps)."""
        out = np.zeros(3, dtype=np.int64)
        self._check(lib().vs_get_hybrid_counters(self._h, _ptr(out)))
        return {"learned_steps": int(out[0]), "fallback_steps": int(out[1]), "exact_vesicles": int(out[2])}

    def profile(self, enable):
        self._check(lib().vs_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} recorded since profile(True)."""
        out = {}
        buf = ctypes.create_string_buffer(128)
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        i = 0
        while lib().vs_profile_read(self._h, i, buf, 128, ctypes.byref(ms), ctypes.byref(n)) == 0:
            out[buf.value.decode()] = (ms.value, n.value)
            i += 1
        return out

    def set_network(self, net, out_scale, filter_kmax, which=0):
        self._net = net  # the library borrows it
        self._check(lib().vs_set_network(self._h, int(which), net._h if net is not None else None, float(out_scale),
                                         int(filter_kmax)))

    def set_gmres(self, tol=1e-10, restart=30, max_iter=300):
        """GMRES settings of the fully implicit step (mode 2, vs_set_gmres)."""
        self._check(lib().vs_set_gmres(self._h, float(tol), int(restart), int(max_iter)))

    def gmres_stats(self):
        """(iterations of the last step, its relative residual estimate, iterations over all steps)."""
        it, tot = ctypes.c_int32(), ctypes.c_int64()
        res = ctypes.c_double()
        self._check(lib().vs_gmres_stats(self._h, ctypes.byref(it), ctypes.byref(res), ctypes.byref(tot)))
        return it.value, res.value, tot.value

    def set_flow_networks(self, adv, ten, Kf, Kout):
        """Learned advection and tension (vs_set_flow_networks); None, None removes them."""
        self._flow = (adv, ten)  # the library borrows them
        self._check(lib().vs_set_flow_networks(self._h, adv._h if adv is not None else None,
                                               ten._h if ten is not None else None, int(Kf), int(Kout)))

    def flow_maps(self, Kf, Kout, filter_kmax, xin_dev, adv_dev, ten_dev):
        """Training rows of the advection and tension networks at the current points (vs_flow_maps)."""
        self._check(lib().vs_flow_maps(self._h, int(Kf), int(Kout), int(filter_kmax), _ptr(xin_dev), _ptr(adv_dev),
                                       _ptr(ten_dev)))

    def set_near_networks(self, nets, Kf, Kout):
        """Learned near-field layers (vs_set_near_networks): five networks, layer order -h .. h; None removes."""
        if nets is None:
            self._near = None
            self._check(lib().vs_set_near_networks(self._h, None, 0, int(Kf), int(Kout)))
            return
        self._near = list(nets)  # the library borrows them
        arr = (ctypes.c_void_p * len(nets))(*[n._h.value for n in nets])
        self._check(lib().vs_set_near_networks(self._h, arr, len(nets), int(Kf), int(Kout)))

    def near_maps(self, Kf, Kout, filter_kmax, xin_dev, out_dev):
        """Training rows of the near-field networks at the current points (vs_near_maps): out_dev holds
        5 x M x flow_adv_width(Kf, Kout) floats, layer-major."""
        self._check(lib().vs_near_maps(self._h, int(Kf), int(Kout), int(filter_kmax), _ptr(xin_dev), _ptr(out_dev)))

    def relax(self, xy_in_dev, xy_out_dev):
        self._check(lib().vs_relax(self._h, _ptr(xy_in_dev), _ptr(xy_out_dev)))

    def training_pairs(self, xy_in_dev, xin_dev, yout_dev, out_scale, filter_kmax):
        self._check(lib().vs_training_pairs(self._h, _ptr(xy_in_dev), _ptr(xin_dev), _ptr(yout_dev), float(out_scale),
                                            int(filter_kmax)))

    def checkpoint(self):
        """The suspension's checkpoint (vs_checkpoint) as bytes."""
        n = ctypes.c_int64()
        self._check(lib().vs_checkpoint_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(lib().vs_checkpoint(self._h, buf, n.value))
        return buf.raw

    def restore(self, data):
        """Load a checkpoint made by checkpoint() (vs_restore)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check(lib().vs_restore(self._h, buf, len(data)))

    def device_ptrs(self):
        a, b = ctypes.c_void_p(), ctypes.c_void_p()
        self._check(lib().vs_get_device_ptrs(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if self._h:
            lib().vs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FarFieldPlan:
    """vs_farfield_plan: far-field single layer of given densities at every point."""

    def __init__(self, offsets, mu=1.0, near_mask=False, precision=0, stream=None):
        L = lib()
        self._h = ctypes.c_void_p()
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        st = L.vs_farfield_plan_create(_ptr(off), len(off) - 1, float(mu), 1 if near_mask else 0, int(precision),
                                       _stream(stream), ctypes.byref(self._h))
        if st != 0:
            raise VsError(st, L.vs_farfield_last_error(None).decode())

    def eval(self, xy, f, u):
        """xy, f, u: device tensors (float64, CSR blocks). u is overwritten."""
        st = lib().vs_farfield_eval(self._h, _ptr(xy), _ptr(f), _ptr(u))
        if st != 0:
            raise VsError(st, lib().vs_farfield_last_error(self._h).decode())

    def counters(self):
        out = np.zeros(2, dtype=np.int64)
        st = lib().vs_farfield_counters(self._h, _ptr(out))
        if st != 0:
            raise VsError(st, lib().vs_farfield_last_error(self._h).decode())
        return {"err": int(out[0]), "near_pairs": int(out[1])}

    def close(self):
        if self._h:
            lib().vs_farfield_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def self_matrices(xy_dev, offsets, mu, out_dev, stream=None):
    """vs_self_matrices: xy_dev / out_dev device tensors (float64)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    st = lib().vs_self_matrices(_ptr(xy_dev), _ptr(off), len(off) - 1, float(mu), _ptr(out_dev), _stream(stream))
    if st != 0:
        raise VsError(st, "vs_self_matrices failed")


def farfield_eval_static(offsets, mu, precision, xy_dev, f_dev, u_dev, stream=None):
    """vs_farfield_eval_static: far field with the library's static scratch (no allocation)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    st = lib().vs_farfield_eval_static(_ptr(off), len(off) - 1, float(mu), int(precision), _ptr(xy_dev),
                                       _ptr(f_dev), _ptr(u_dev), _stream(stream))
    if st != 0:
        raise VsError(st, "vs_farfield_eval_static failed")


class VsAdamW(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("weight_decay", ctypes.c_float)]


def batched_inverse32(a_dev, out_dev, n, batch, stream=None):
    """vs_batched_inverse32 on device FP32 tensors; returns the number of pivoting fallbacks."""
    fb = ctypes.c_int32()
    st = lib().vs_batched_inverse32(_ptr(a_dev), _ptr(out_dev), int(n), int(batch), ctypes.byref(fb), _stream(stream))
    if st != 0:
        raise VsError(st, "vs_batched_inverse32 failed")
    return fb.value


def fp32_rate(mix, iters=2048, stream=None):
    """vs_fp32_rate: (T FP32 lane-ops/s, ms) of the register-only probe (mix 0 paired FMA chains, mix 1 the far
    field's paired pair arithmetic)."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    st = lib().vs_fp32_rate(int(mix), int(iters), ctypes.byref(r), ctypes.byref(ms), _stream(stream))
    if st != 0:
        raise VsError(st, "vs_fp32_rate failed")
    return r.value, ms.value


def flow_widths(Kf, Kout):
    """Output widths (advection, tension) of the flow networks (vs_set_flow_networks)."""
    nb, po = 4 * Kf + 2, 2 * Kout + 1
    return (nb * 2 * po + 15) // 16 * 16, ((nb + 1) * po + 15) // 16 * 16


def feature_width(N, kmax):
    """Width of the relaxation network's feature rows (vs_set_network): 16 ceil((4K + 2)/16),
    K = min(kmax, N/2 - 1)."""
    K = min(int(kmax), int(N) // 2 - 1)
    return (4 * K + 2 + 15) // 16 * 16


class Mlp:
    """vs_mlp: BF16 tensor-core MLP (ReLU hidden layers) with the paper's loss and AdamW."""

    def __init__(self, dims, max_batch, ncomp=2, beta=1.0, stream=None):
        L = lib()
        self._h = ctypes.c_void_p()
        d = np.ascontiguousarray(dims, dtype=np.int32)
        st = L.vs_mlp_create(_ptr(d), len(d) - 1, int(max_batch), int(ncomp), float(beta), _stream(stream),
                             ctypes.byref(self._h))
        if st != 0:
            raise VsError(st, L.vs_mlp_last_error(None).decode())
        n = ctypes.c_int64()
        self._check(L.vs_mlp_num_params(self._h, ctypes.byref(n)))
        self.nparam = n.value
        self.dims = list(dims)

    def _check(self, st):
        if st != 0:
            raise VsError(st, lib().vs_mlp_last_error(self._h).decode())

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().vs_mlp_set_params(self._h, _ptr(p), len(p)))

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        self._check(lib().vs_mlp_get_params(self._h, _ptr(p), len(p)))
        return p

    def set_affine(self, in_shift=None, in_scale=None, out_shift=None, out_scale=None):
        """Per-feature input and output maps (vs_mlp_set_affine); None is the identity part."""
        arr = [None if a is None else np.ascontiguousarray(a, dtype=np.float32)
               for a in (in_shift, in_scale, out_shift, out_scale)]
        for a, d in zip(arr, (self.dims[0], self.dims[0], self.dims[-1], self.dims[-1])):
            if a is not None and a.shape != (d,):
                raise ValueError("affine map of width %d expected" % d)
        self._check(lib().vs_mlp_set_affine(self._h, *[None if a is None else _ptr(a) for a in arr]))

    def get_affine(self):
        """(in_shift, in_scale, out_shift, out_scale) as FP32 host arrays."""
        d0, dL = self.dims[0], self.dims[-1]
        out = [np.empty(d0, np.float32), np.empty(d0, np.float32), np.empty(dL, np.float32),
               np.empty(dL, np.float32)]
        self._check(lib().vs_mlp_get_affine(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def fit_affine(self, x_dev, y_dev, rows, rel_floor=0.0):
        """Maps from the column means and deviations of device rows x, y (vs_mlp_fit_affine)."""
        self._check(lib().vs_mlp_fit_affine(self._h, _ptr(x_dev), _ptr(y_dev), int(rows), float(rel_floor)))

    def forward(self, x_dev, y_dev, batch):
        self._check(lib().vs_mlp_forward(self._h, _ptr(x_dev), int(batch), _ptr(y_dev)))

    def loss_grad(self, x_dev, y_dev, batch, want_grad=True):
        loss = ctypes.c_float()
        g = np.empty(self.nparam, dtype=np.float32) if want_grad else None
        self._check(lib().vs_mlp_loss_grad(self._h, _ptr(x_dev), _ptr(y_dev), int(batch), ctypes.byref(loss),
                                           _ptr(g) if want_grad else None, self.nparam))
        return loss.value, g

    def train_step(self, x_dev, y_dev, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01,
                   want_loss=False):
        opt = VsAdamW(lr, beta1, beta2, eps, weight_decay)
        loss = ctypes.c_float()
        self._check(lib().vs_mlp_train_step(self._h, _ptr(x_dev), _ptr(y_dev), int(batch), ctypes.byref(opt),
                                            ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def sync(self):
        self._check(lib().vs_mlp_sync(self._h))

    def close(self):
        if self._h:
            lib().vs_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ivnet:
    """vs_ivnet: the paper's IVNet (Sec. 3.4.2) on the BF16 tensor-core GEMMs, with the paper's loss and AdamW.
    Samples are rows [x(N), y(N)]."""

    def __init__(self, N, C, nblocks, max_batch, beta=1.0, stream=None, in_channels=2):
        L = lib()
        self._h = ctypes.c_void_p()
        st = L.vs_ivnet_create(int(N), int(in_channels), int(C), int(nblocks), int(max_batch), float(beta),
                               _stream(stream), ctypes.byref(self._h))
        if st != 0:
            raise VsError(st, L.vs_ivnet_last_error(None).decode())
        n = ctypes.c_int64()
        self._check(L.vs_ivnet_num_params(self._h, ctypes.byref(n)))
        self.nparam = n.value
        self.N, self.C, self.nblocks, self.in_channels = N, C, nblocks, in_channels

    def _check(self, st):
        if st != 0:
            raise VsError(st, lib().vs_ivnet_last_error(self._h).decode())

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().vs_ivnet_set_params(self._h, _ptr(p), len(p)))

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        self._check(lib().vs_ivnet_get_params(self._h, _ptr(p), len(p)))
        return p

    def set_affine(self, in_shift=None, in_scale=None, out_shift=None, out_scale=None):
        arr = [None if a is None else np.ascontiguousarray(a, dtype=np.float32)
               for a in (in_shift, in_scale, out_shift, out_scale)]
        for a, d in zip(arr, (self.in_channels, self.in_channels, 2, 2)):
            if a is not None and a.shape != (d * self.N,):
                raise ValueError("affine map of width %d expected" % (d * self.N))
        self._check(lib().vs_ivnet_set_affine(self._h, *[None if a is None else _ptr(a) for a in arr]))

    def fit_affine(self, x_dev, y_dev, rows, rel_floor=0.0):
        self._check(lib().vs_ivnet_fit_affine(self._h, _ptr(x_dev), _ptr(y_dev), int(rows), float(rel_floor)))

    def forward(self, x_dev, y_dev, batch):
        self._check(lib().vs_ivnet_forward(self._h, _ptr(x_dev), int(batch), _ptr(y_dev)))

    def loss_grad(self, x_dev, y_dev, batch, want_grad=True):
        loss = ctypes.c_float()
        g = np.empty(self.nparam, dtype=np.float32) if want_grad else None
        self._check(lib().vs_ivnet_loss_grad(self._h, _ptr(x_dev), _ptr(y_dev), int(batch), ctypes.byref(loss),
                                             _ptr(g) if want_grad else None, self.nparam))
        return loss.value, g

    def train_step(self, x_dev, y_dev, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01,
                   want_loss=False):
        opt = VsAdamW(lr, beta1, beta2, eps, weight_decay)
        loss = ctypes.c_float()
        self._check(lib().vs_ivnet_train_step(self._h, _ptr(x_dev), _ptr(y_dev), int(batch), ctypes.byref(opt),
                                              ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def sync(self):
        self._check(lib().vs_ivnet_sync(self._h))

    def close(self):
        if self._h:
            lib().vs_ivnet_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def feature_points(feat_dev, rows, ld, N, K, out_dev, stream=None):
    """vs_feature_points: samples [x(N), y(N)] of Fourier feature rows (device FP32)."""
    st = lib().vs_feature_points(_ptr(feat_dev), int(rows), int(ld), int(N), int(K), _ptr(out_dev), _stream(stream))
    if st != 0:
        raise VsError(st, "vs_feature_points failed")


def standardize(xy_dev, offsets, kmax, xin_dev, frames_dev, stream=None):
    """vs_standardize: FP32 network input rows and frames of every vesicle (device tensors)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    st = lib().vs_standardize(_ptr(xy_dev), _ptr(off), len(off) - 1, int(kmax), _ptr(xin_dev), _ptr(frames_dev),
                              _stream(stream))
    if st != 0:
        raise VsError(st, "vs_standardize failed")
