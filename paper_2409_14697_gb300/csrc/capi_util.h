// Helpers shared by the C entry points: error translation into return codes.
#pragma once

#include <new>
#include <stdexcept>
#include <string>

#include "qs_internal.h"

namespace qs {
extern thread_local std::string g_last_error;
}

#define QS_API_BEGIN try {
#define QS_API_END                                  \
    }                                               \
    catch (const qs::Error &e) {                    \
        qs::g_last_error = e.msg;                   \
        return e.code;                              \
    }                                               \
    catch (const std::bad_alloc &) {                \
        qs::g_last_error = "host allocation failed"; \
        return QS_ERR_NOMEM;                        \
    }                                               \
    catch (const std::exception &e) {               \
        qs::g_last_error = e.what();                \
        return QS_ERR_CUDA;                         \
    }                                               \
    qs::g_last_error.clear();                       \
    return QS_OK;


// As QS_API_END, but returns rc (e.g. QS_NOT_READY) on success.
#define QS_API_END_RC(rc)                           \
    }                                               \
    catch (const qs::Error &e) {                    \
        qs::g_last_error = e.msg;                   \
        return e.code;                              \
    }                                               \
    catch (const std::bad_alloc &) {                \
        qs::g_last_error = "host allocation failed"; \
        return QS_ERR_NOMEM;                        \
    }                                               \
    catch (const std::exception &e) {               \
        qs::g_last_error = e.what();                \
        return QS_ERR_CUDA;                         \
    }                                               \
    qs::g_last_error.clear();                       \
    return (rc);
