"""Python binding of the C ABI (include/lbm.h), one function per entry point
with the same name.  It only marshals arguments: numpy arrays in, numpy arrays
out; every step of the method runs in the CUDA library."""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_float, c_int64, c_uint8, c_void_p

import numpy as np

from . import _lib, _torch_alloc
from ._lib import LbmConfig, LbmMlp, LbmTrainOpts
from ._torch_alloc import use_torch_allocator  # noqa: F401

LBM_BGK, LBM_MRT = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16DEV = 0, 1, 2
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16dev": LBM_FP16DEV}
COLLISIONS = {"bgk": LBM_BGK, "mrt": LBM_MRT}


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_lib.STATUS.get(status, status)}: {message}")
        self.status = status


def _check(st):
    if st != 0:
        msg = _lib.load().lbm_last_error().decode(errors="replace")
        raise LbmError(st, msg)


def _dptr(a):
    return a.ctypes.data_as(POINTER(c_double))


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


class Sim:
    """Handle of a simulation created by lbm_create."""

    def __init__(self, handle, cfg):
        self.handle = handle
        self.nx, self.ny = cfg.nx, cfg.ny
        self.cfg = cfg
        _torch_alloc.track(self)

    def close(self):
        if self.handle:
            _lib.load().lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_set_default_allocator(alloc):
    """Install an LbmAllocator (a ctypes struct whose callbacks the caller
    keeps alive) as the library's default device allocator; None restores
    cudaMalloc / cudaFree.  The binding installs torch's caching allocator on
    load (see use_torch_allocator)."""
    _check(_lib.load().lbm_set_default_allocator(byref(alloc) if alloc is not None else None))


def lbm_config_default(**kw):
    """Default lbm_config with the given fields set (collision "bgk"/"mrt", precision
    "fp64"/"fp32"/"fp16dev", layout "ab"/"aa", stream a CUDA stream handle or 0)."""
    cfg = LbmConfig()
    _check(_lib.load().lbm_config_default(byref(cfg)))
    for k, v in kw.items():
        if k == "collision" and isinstance(v, str):
            v = COLLISIONS[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "layout" and isinstance(v, str):
            v = {"ab": 0, "aa": 1}[v]
        if k == "mrt_rates":
            arr = (c_double * 9)(*[float(r) for r in v])
            cfg.mrt_rates = arr
            continue
        if k == "stream":
            v = c_void_p(int(v)) if v else None
        setattr(cfg, k, v)
    return cfg


def lbm_create(cfg):
    """Create a simulation from a config; returns a Sim handle."""
    h = c_void_p()
    _check(_lib.load().lbm_create(byref(cfg), byref(h)))
    return Sim(h, cfg)


def lbm_destroy(sim):
    """Destroy a simulation (fails while a batch holds it)."""
    if sim.handle:
        _check(_lib.load().lbm_destroy(sim.handle))
        sim.handle = None


def lbm_set_geometry(sim, kind):
    """Cell kinds, uint8 of shape (ny, nx): 0 fluid, 1 solid body (its links count in
    the force), 2 wall (solid, not counted)."""
    k = np.ascontiguousarray(kind, dtype=np.uint8)
    if k.shape != (sim.ny, sim.nx):
        raise ValueError("kind must have shape (ny, nx)")
    _check(_lib.load().lbm_set_geometry(sim.handle, k.ctypes.data_as(POINTER(c_uint8))))


def lbm_init_equilibrium(sim, rho=None, ux=None, uy=None):
    """Populations f_eq(rho, u) from (ny, nx) fields; None means rho = 1, u = 0.
    Resets the step counter, the force series and the boundary state."""
    shape = (sim.ny, sim.nx)
    arrs = [None if a is None else _f64(a, shape) for a in (rho, ux, uy)]
    ptrs = [None if a is None else _dptr(a) for a in arrs]
    _check(_lib.load().lbm_init_equilibrium(sim.handle, *ptrs))


def lbm_set_outflow_zouhe(sim, rho_out=1.0):
    """Zou & He pressure outflow at x = nx - 1 with density rho_out."""
    _check(_lib.load().lbm_set_outflow_zouhe(sim.handle, float(rho_out)))


def make_mlp(layers, act="tanh", in_mean=None, in_std=None, out_scale=1.0):
    """Marshal a network given as [(W (n_out, n_in), b), ...] into an LbmMlp.
    Returns (struct, keepalive) -- keep the second alive while the struct is used."""
    if len(layers) > _lib.MLP_MAX_LAYERS:
        raise ValueError("at most 4 layers")
    sizes = [int(np.shape(layers[0][0])[1])] + [int(np.shape(W)[0]) for W, _ in layers]
    flat = np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(),
                                           np.asarray(b, np.float32).ravel()]) for W, b in layers])
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    m = LbmMlp()
    m.n_layers = len(layers)
    for l in range(_lib.MLP_MAX_LAYERS + 1):
        m.sizes[l] = sizes[l] if l < len(sizes) else 0
    m.act = {"tanh": 0, "leaky": 1}[act] if isinstance(act, str) else int(act)
    m.params = flat.ctypes.data_as(POINTER(c_float))
    m.n_params = flat.size
    keep = [flat]
    if in_mean is not None:
        a = np.ascontiguousarray(in_mean, dtype=np.float32)
        keep.append(a)
        m.in_mean = a.ctypes.data_as(POINTER(c_float))
    if in_std is not None:
        a = np.ascontiguousarray(in_std, dtype=np.float32)
        keep.append(a)
        m.in_std = a.ctypes.data_as(POINTER(c_float))
    m.out_scale = float(out_scale)
    return m, keep


def lbm_set_outflow_nn(sim, layers, act="tanh", in_mean=None, in_std=None, out_scale=1.0,
                       fallback_drho=0.05):
    m, keep = make_mlp(layers, act, in_mean, in_std, out_scale)
    _check(_lib.load().lbm_set_outflow_nn(sim.handle, byref(m), float(fallback_drho)))
    del keep


def lbm_set_outflow_cbc(sim, sigma=0.0, kappa2=0.0, mach=0.0, length=0.0, tuner=None,
                        act="leaky", in_mean=None, in_std=None, exact_mass=False):
    """Characteristic outflow; ``tuner`` is [(W, b), ...] mapping 6 -> 1 or 2."""
    keep = None
    m = None
    if tuner is not None:
        m, keep = make_mlp(tuner, act, in_mean, in_std, 1.0)
    _check(_lib.load().lbm_set_outflow_cbc(sim.handle, float(sigma), float(kappa2), float(mach),
                                           float(length), byref(m) if m is not None else None,
                                           int(bool(exact_mass))))
    del keep


def lbm_nn_fallbacks(sim):
    """Number of network-outflow nodes that fell back to Zou & He so far."""
    c = c_int64()
    _check(_lib.load().lbm_nn_fallbacks(sim.handle, byref(c)))
    return c.value


def _devptr(buf):
    """Device address of a CUDA tensor (or a raw address given as an int)."""
    if isinstance(buf, int):
        return buf
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return buf.data_ptr()


def lbm_capture_plane(sim, x_t, every, rows=None, cap_rows=None):
    """Capture training rows at column x_t every ``every`` steps into ``rows``
    (a contiguous float32 CUDA tensor of shape (cap_rows, 84)); rows=None stops."""
    if rows is None:
        _check(_lib.load().lbm_capture_plane(sim.handle, 0, 0, None, 0))
        return
    if cap_rows is None:
        cap_rows = rows.shape[0]
    _check(_lib.load().lbm_capture_plane(sim.handle, int(x_t), int(every),
                                         c_void_p(_devptr(rows)), int(cap_rows)))


def lbm_capture_snapshot(sim, x_begin, x_end, rows):
    """Rows of the columns [x_begin, x_end) of the current state into the device
    tensor ``rows`` ((x_end - x_begin) * ny, 84), one batch of ny rows per column."""
    need = (int(x_end) - int(x_begin)) * sim.ny
    if rows.shape[0] < need or rows.shape[1] != 84:
        raise ValueError(f"rows must hold {need} x 84 floats")
    _check(_lib.load().lbm_capture_snapshot(sim.handle, int(x_begin), int(x_end),
                                            c_void_p(_devptr(rows))))


def lbm_save(sim, path):
    """Write a checkpoint (populations and step counter) to a file."""
    _check(_lib.load().lbm_save(sim.handle, str(path).encode()))


def lbm_load(sim, path):
    """Read a checkpoint written by lbm_save for a sim of the same size and precision."""
    _check(_lib.load().lbm_load(sim.handle, str(path).encode()))


def lbm_capture_count(sim):
    """Rows written so far by lbm_capture_plane."""
    c = c_int64()
    _check(_lib.load().lbm_capture_count(sim.handle, byref(c)))
    return c.value


def lbm_nn_dataset_stats(rows, n_rows=None, stream=None):
    """(in_mean[81], in_std[81], out_scale) of a device data set of rows."""
    n = rows.shape[0] if n_rows is None else n_rows
    mean = np.zeros(81, np.float32)
    std = np.zeros(81, np.float32)
    scale = c_float()
    _check(_lib.load().lbm_nn_dataset_stats(c_void_p(_devptr(rows)), int(n),
                                            c_void_p(int(stream)) if stream else None,
                                            mean.ctypes.data_as(POINTER(c_float)),
                                            std.ctypes.data_as(POINTER(c_float)), byref(scale)))
    return mean, std, scale.value


def lbm_train_opts_default(**kw):
    """Default training options with the given fields set."""
    o = LbmTrainOpts()
    _check(_lib.load().lbm_train_opts_default(byref(o)))
    for k, v in kw.items():
        if k == "stream":
            v = c_void_p(int(v)) if v else None
        setattr(o, k, v)
    return o


def _order(order):
    return np.ascontiguousarray(order, dtype=np.int32)


def lbm_nn_train(rows, order, layers, act="tanh", in_mean=None, in_std=None, out_scale=1.0,
                 adam_m=None, adam_v=None, n_rows=None, **opts):
    """Adam steps of Eq. 16 on device rows, batch order[k] at step k.
    Returns (layers, adam_m, adam_v, losses) with the trained layers as float32."""
    o = lbm_train_opts_default(**opts)
    m, keep = make_mlp(layers, act, in_mean, in_std, out_scale)
    order = _order(order)
    n = rows.shape[0] if n_rows is None else n_rows
    out = np.zeros(m.n_params, np.float32)
    am = np.zeros(m.n_params, np.float32) if adam_m is None else \
        np.ascontiguousarray(adam_m, dtype=np.float32).copy()
    av = np.zeros(m.n_params, np.float32) if adam_v is None else \
        np.ascontiguousarray(adam_v, dtype=np.float32).copy()
    losses = np.zeros(order.size, np.float64)
    _check(_lib.load().lbm_nn_train(c_void_p(_devptr(rows)), int(n),
                                    order.ctypes.data_as(POINTER(ctypes.c_int32)), order.size,
                                    byref(o), byref(m), out.ctypes.data_as(POINTER(c_float)),
                                    am.ctypes.data_as(POINTER(c_float)),
                                    av.ctypes.data_as(POINTER(c_float)), _dptr(losses)))
    del keep
    return unflatten(out, layers), am, av, losses


def lbm_nn_loss_grad(rows, order, layers, act="tanh", in_mean=None, in_std=None, out_scale=1.0,
                     grads=True, n_rows=None, **opts):
    """Loss of Eq. 16 per listed batch and (grads=True) the flat gradients,
    shape (n_batches, n_params), in the parameter layout of make_mlp."""
    o = lbm_train_opts_default(**opts)
    m, keep = make_mlp(layers, act, in_mean, in_std, out_scale)
    order = _order(order)
    n = rows.shape[0] if n_rows is None else n_rows
    losses = np.zeros(order.size, np.float64)
    g = np.zeros((order.size, m.n_params), np.float32) if grads else None
    _check(_lib.load().lbm_nn_loss_grad(c_void_p(_devptr(rows)), int(n),
                                        order.ctypes.data_as(POINTER(ctypes.c_int32)),
                                        order.size, byref(o), byref(m), _dptr(losses),
                                        g.ctypes.data_as(POINTER(c_float)) if grads else None))
    del keep
    return (losses, g) if grads else losses


def lbm_copy_columns(sim, x0, width, out):
    """Populations f (FP64, not shifted) of columns [x0, x0 + width) into the
    device tensor ``out`` (9, ny, width), enqueued on the sim's stream."""
    _check(_lib.load().lbm_copy_columns(sim.handle, int(x0), int(width), c_void_p(_devptr(out))))


def _segments(bank, nx, n_t, tau, sigma, kappa2, mach, init_state, final_state, length=0.0,
              rho_out=1.0, exact_mass=False, precision="fp64", stream=None):
    """LbmCbcSegments over a device bank (n_states, 9, ny, bank_width) float64."""
    n_states, _, ny, width = (int(d) for d in bank.shape)
    init = np.ascontiguousarray(init_state, dtype=np.int32)
    fin = np.ascontiguousarray(final_state, dtype=np.int32)
    if init.shape != fin.shape:
        raise ValueError("init_state and final_state differ in length")
    g = _lib.LbmCbcSegments()
    g.nx, g.ny, g.n_t = int(nx), ny, int(n_t)
    g.tau, g.rho_out = float(tau), float(rho_out)
    g.sigma, g.kappa2, g.mach, g.length = float(sigma), float(kappa2), float(mach), float(length)
    g.exact_mass = int(bool(exact_mass))
    g.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    g.bank = c_void_p(_devptr(bank))
    g.n_states, g.bank_width = n_states, width
    g.init_state = init.ctypes.data_as(POINTER(ctypes.c_int32))
    g.final_state = fin.ctypes.data_as(POINTER(ctypes.c_int32))
    g.n_seg = int(init.size)
    g.stream = c_void_p(int(stream)) if stream else None
    return g, [init, fin]


def lbm_cbc_feature_stats(bank, stream=None):
    """(in_mean[6], in_std[6]) of the tuner's features over every bank state."""
    g, keep = _segments(bank, int(bank.shape[3]) + 1, 1, 0.6, 0.0, 0.0, 0.0, [0], [0],
                        stream=stream)
    mean = np.zeros(6, np.float32)
    std = np.zeros(6, np.float32)
    _check(_lib.load().lbm_cbc_feature_stats(byref(g), mean.ctypes.data_as(POINTER(c_float)),
                                             std.ctypes.data_as(POINTER(c_float))))
    del keep
    return mean, std


def _tuner_struct(tuner, act, in_mean, in_std):
    m, keep = make_mlp(tuner, act, in_mean, in_std, 1.0)
    flat = np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(),
                                           np.asarray(b, np.float64).ravel()]) for W, b in tuner])
    return m, keep, np.ascontiguousarray(flat)


def lbm_cbc_segment_grad(bank, nx, n_t, tau, sigma, kappa2, mach, init_state, final_state, tuner,
                         act="leaky", in_mean=None, in_std=None, params=None, grad=True, **kw):
    """Mean segment loss and (grad=True) its flat FP64 gradient with respect to
    the tuner's parameters, evaluated at ``params`` (flat float64, default the
    tuner's own values in float64)."""
    g, keep_g = _segments(bank, nx, n_t, tau, sigma, kappa2, mach, init_state, final_state, **kw)
    m, keep, flat = _tuner_struct(tuner, act, in_mean, in_std)
    p = flat if params is None else np.ascontiguousarray(params, dtype=np.float64)
    loss = np.zeros(1)
    gr = np.zeros(p.size) if grad else None
    _check(_lib.load().lbm_cbc_segment_grad(byref(g), byref(m), _dptr(p), _dptr(loss),
                                            _dptr(gr) if grad else None))
    del keep, keep_g
    return (float(loss[0]), gr) if grad else float(loss[0])


def lbm_cbc_tuner_train(bank, nx, n_t, tau, sigma, kappa2, mach, init_state, final_state, tuner,
                        order, batch, act="leaky", in_mean=None, in_std=None, params=None,
                        adam_m=None, adam_v=None, lr=1e-3, adam_t0=0, stream=None, **kw):
    """Adam steps on the segment loss, batch k = segments order[k*batch:(k+1)*batch].
    Returns (params, adam_m, adam_v, losses), all float64."""
    g, keep_g = _segments(bank, nx, n_t, tau, sigma, kappa2, mach, init_state, final_state,
                          stream=stream, **kw)
    m, keep, flat = _tuner_struct(tuner, act, in_mean, in_std)
    p = (flat if params is None else np.asarray(params, np.float64)).copy()
    am = np.zeros(p.size) if adam_m is None else np.asarray(adam_m, np.float64).copy()
    av = np.zeros(p.size) if adam_v is None else np.asarray(adam_v, np.float64).copy()
    order = _order(order)
    n_steps = order.size // int(batch) if int(batch) > 0 else 0
    losses = np.zeros(n_steps)
    o = lbm_train_opts_default(lr=float(lr), adam_t0=int(adam_t0), stream=stream)
    _check(_lib.load().lbm_cbc_tuner_train(byref(g), byref(m),
                                           order.ctypes.data_as(POINTER(ctypes.c_int32)),
                                           int(batch), n_steps, byref(o), _dptr(p), _dptr(am),
                                           _dptr(av), _dptr(losses)))
    del keep, keep_g
    return p, am, av, losses


def unflatten(flat, like):
    """Split a flat parameter vector into [(W, b), ...] shaped like ``like``."""
    out, off = [], 0
    for W, b in like:
        nw, nb = int(np.size(W)), int(np.size(b))
        out.append((np.asarray(flat[off:off + nw]).reshape(np.shape(W)),
                    np.asarray(flat[off + nw:off + nw + nb])))
        off += nw + nb
    return out


def lbm_step(sim, n=1):
    """Enqueue n time steps on the sim's stream (returns at once)."""
    _check(_lib.load().lbm_step(sim.handle, int(n)))


def lbm_sync(sim):
    """Wait for the sim's stream; raises LbmError for a latched device fault."""
    _check(_lib.load().lbm_sync(sim.handle))


def lbm_time(sim):
    """Step counter (time steps taken since the last initialisation or load)."""
    t = c_int64()
    _check(_lib.load().lbm_time(sim.handle, byref(t)))
    return t.value


def lbm_forces(sim, cap=None):
    """Drain the force series: returns (fx, fy) arrays."""
    if cap is None:
        cap = max(lbm_time(sim), 1)
    fx = np.empty(cap)
    fy = np.empty(cap)
    n = c_int64()
    _check(_lib.load().lbm_forces(sim.handle, _dptr(fx), _dptr(fy), int(cap), byref(n)))
    return fx[:n.value].copy(), fy[:n.value].copy()


def lbm_fields(sim):
    """Macroscopic fields: (rho, ux, uy), each float64 of shape (ny, nx)."""
    rho = np.empty((sim.ny, sim.nx))
    ux = np.empty((sim.ny, sim.nx))
    uy = np.empty((sim.ny, sim.nx))
    _check(_lib.load().lbm_fields(sim.handle, _dptr(rho), _dptr(ux), _dptr(uy)))
    return rho, ux, uy


def lbm_get_populations(sim):
    """Populations f_i(x, y) as float64 of shape (9, ny, nx)."""
    f = np.empty((9, sim.ny, sim.nx))
    _check(_lib.load().lbm_get_populations(sim.handle, _dptr(f)))
    return f


def lbm_set_populations(sim, f):
    """Replace the populations by a float64 array of shape (9, ny, nx)."""
    f = _f64(f, (9, sim.ny, sim.nx))
    _check(_lib.load().lbm_set_populations(sim.handle, _dptr(f)))


def lbm_mass(sim):
    """Total mass (sum of rho over fluid nodes, FP64)."""
    m = c_double()
    _check(_lib.load().lbm_mass(sim.handle, byref(m)))
    return m.value


def lbm_device_state(sim):
    """Zero-copy view of the current populations: (device address, pitch, plane)
    in elements of the storage type (see lbm.h for the layout)."""
    base = c_void_p()
    pitch = c_int64()
    plane = c_int64()
    _check(_lib.load().lbm_device_state(sim.handle, byref(base), byref(pitch), byref(plane)))
    return base.value, pitch.value, plane.value


def lbm_set_tiling(sim, rows, variant):
    """Strip height (rows) and kernel variant of the sim's own step launch (see lbm.h)."""
    _check(_lib.load().lbm_set_tiling(sim.handle, int(rows), int(variant)))


def lbm_debug_hold_dataflow(sim, hold):
    """Test hook: make the dataflow variant's flag waits run out (see lbm.h)."""
    _check(_lib.load().lbm_debug_hold_dataflow(sim.handle, int(hold)))


def lbm_get_tiling(sim):
    """Returns (rows, variant) of the sim's own step launch."""
    r = ctypes.c_int32()
    v = ctypes.c_int32()
    _check(_lib.load().lbm_get_tiling(sim.handle, byref(r), byref(v)))
    return r.value, v.value


def lbm_autotune(sim, steps=20, flush_bytes=0):
    """Returns (rows, variant, mean step ms) of the fastest tiling, now in use."""
    ms = c_float()
    _check(_lib.load().lbm_autotune(sim.handle, int(steps), int(flush_bytes), byref(ms)))
    r, v = lbm_get_tiling(sim)
    return r, v, ms.value


def lbm_step_noalloc(cfg, src_ptr, dst_ptr, kind_ptr, pitch, t, force_ptr):
    """One step on caller-owned device buffers (raw device pointers as ints);
    the library allocates nothing.  See include/lbm.h."""
    _check(_lib.load().lbm_step_noalloc(byref(cfg), c_void_p(src_ptr), c_void_p(dst_ptr),
                                        c_void_p(kind_ptr), int(pitch), int(t),
                                        c_void_p(force_ptr)))


class Batch:
    """Handle of a batch created by lbm_batch_create (keeps its members alive)."""

    def __init__(self, handle, sims):
        self.handle = handle
        self.sims = list(sims)
        _torch_alloc.track(self)

    def close(self):
        if self.handle:
            _lib.load().lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_batch_create(sims):
    """Batch of sims of one precision and stream, advanced together; returns a Batch."""
    arr = (c_void_p * len(sims))(*[s.handle.value if isinstance(s.handle, c_void_p) else s.handle
                                   for s in sims])
    h = c_void_p()
    _check(_lib.load().lbm_batch_create(arr, len(sims), byref(h)))
    return Batch(h, sims)


def lbm_batch_destroy(batch):
    """Destroy a batch (its sims stay valid)."""
    if batch.handle:
        _check(_lib.load().lbm_batch_destroy(batch.handle))
        batch.handle = None


def lbm_batch_step(batch, n=1):
    """Enqueue n time steps of every member (one launch per step)."""
    _check(_lib.load().lbm_batch_step(batch.handle, int(n)))


def lbm_batch_sync(batch):
    """Wait for the batch's stream; raises LbmError for a latched fault of any member."""
    _check(_lib.load().lbm_batch_sync(batch.handle))


def lbm_batch_set_tiling(batch, rows, variant):
    """Strip height and kernel variant of the batch launch."""
    _check(_lib.load().lbm_batch_set_tiling(batch.handle, int(rows), int(variant)))


def lbm_batch_get_tiling(batch):
    """Returns (rows, variant) of the batch launch."""
    r = ctypes.c_int32()
    v = ctypes.c_int32()
    _check(_lib.load().lbm_batch_get_tiling(batch.handle, byref(r), byref(v)))
    return r.value, v.value


def lbm_batch_autotune(batch, steps=20, flush_bytes=0):
    """Returns (rows, variant, mean step ms) of the fastest batch tiling, now in use."""
    ms = c_float()
    _check(_lib.load().lbm_batch_autotune(batch.handle, int(steps), int(flush_bytes), byref(ms)))
    r, v = lbm_batch_get_tiling(batch)
    return r, v, ms.value


def lbm_strouhal(cl, length, u):
    """Strouhal number of a lift-coefficient series (dominant frequency x length / u)."""
    cl = np.ascontiguousarray(cl, dtype=np.float64)
    st = c_double()
    _check(_lib.load().lbm_strouhal(_dptr(cl), cl.size, float(length), float(u), byref(st)))
    return st.value


def lbm_version():
    """Version string of the library."""
    return _lib.load().lbm_version().decode()
